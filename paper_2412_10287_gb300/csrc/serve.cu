// Serving: continuous batching of single-source queries over the lane engine.
//
// The paper runs queries one at a time (section 5.3).  A server instead keeps
// the graph and the state of every admitted query resident on the device and
// lets queries that arrive while others run join at the next level boundary:
//
//   loop
//     admit    queued queries take free lanes (one bit of the 256-lane vector
//              per query; automaton state q in slot q); their source is
//              seeded into the current frontier and the visited set;
//     step     one level of Algorithm 1 for every lane at once: the captured
//              CUDA graph of the lane step (expand frontier rows, expand long
//              row chunks, commit, read back the lanes that found new pairs);
//     retire   a lane whose frontier is now empty (or that reached the level
//              cap) is finished: one pass over the visited set extracts the
//              answers of all finishing lanes and clears their bits, and the
//              lanes become free.
//
// Lanes never interact (every Boolean operation is bitwise per lane), so an
// answer is the same whether the query ran alone or among others.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "lanes.h"

using Clock = std::chrono::steady_clock;

namespace rpq {
namespace {

constexpr size_t kServeTablesBytes = 4u << 20;

struct Pending {
    uint64_t ticket;
    Automaton a;
    int32_t source;
    Clock::time_point t_submit;
};

struct Done {
    rpq_status status = RPQ_OK;
    std::vector<int32_t> answer;
};

struct Lane {
    bool busy = false;
    bool finished = false;
    int64_t bytes = 0;  // device state counted against the memory budget
    uint64_t ticket = 0;
    Automaton a;
    int32_t source = 0;
    int level = 0;
    int64_t finished_step = 0;
    Clock::time_point t_submit;
};

}  // namespace
}  // namespace rpq

struct rpq_server {
    rpq_graph *g = nullptr;
    int engine = 0;
    int lanes_max = 0, K = 0, max_levels = 0;
    std::vector<std::thread> slot_workers;
    size_t queue_cap = 0;
    std::unique_ptr<rpq::LaneWorkspace> ws;
    cudaStream_t st = nullptr;
    cudaGraphExec_t step_exec = nullptr;
    rpq::DevBuf tables, step_out;
    void *staging = nullptr;            // pinned: tables upload
    rpq::LaneStepOut *out_host = nullptr;  // pinned: step read-back
    rpq::LParams p{};
    size_t o_dyn = 0, o_dirs = 0, o_units = 0, o_srcs = 0, o_fm = 0, o_seed = 0, o_verts = 0;

    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::deque<rpq::Pending> queue;
    std::unordered_map<uint64_t, rpq::Done> results;
    std::unordered_map<uint64_t, int> inflight;  // ticket -> 1 (queued or running)
    rpq::Lane lane[rpq::kLanes];
    bool stop = false;
    std::thread worker;
    uint64_t next_ticket = 1;
    // admission: device state of the admitted queries against the budget
    int64_t budget = 0;          // 0 = no limit
    int64_t inflight_bytes = 0, peak_bytes = 0;
    int inflight_n = 0, peak_inflight = 0;
    // engine 0: queries in flight at most, lowered after an allocation
    // failure (back-off) and raised again as queries complete
    int slot_cap = 0;
    int64_t oom_retries = 0;
    // engine 0: a query is launched on 1 / d of the grid, d = 1 + the queries
    // still queued when it is admitted, and at least idle_div (2: at 2,000
    // q/s on rmat20 half the grid for a query that finds the queue empty gave
    // p50 0.16 ms and p99 1.16 ms, the whole grid 0.37 / 1.28 ms; counting
    // the queries in flight into d as well gave 0.13 / 1.23 ms)
    int idle_div = 2;
    // statistics
    int64_t submitted = 0, admitted = 0, completed = 0, rejected = 0, level_steps = 0;
    std::vector<double> latency_ms;
    bool started = false;
    Clock::time_point t_first, t_last;
    rpq_status fatal = RPQ_OK;
};

namespace rpq {
namespace {

// Device state of one admitted query, the unit of memory-bounded
// admission.  Engine 0: the query's workspace -- the visited bitset P and
// three frontier bitsets of S_cap x ceil(n/64) words, and the visited lists of
// S_cap x n ids (S_cap: the state count rounded up to a power of two, at
// least 4, as workspaces are sized).  Engine 1: the query's bits in the four
// lane arrays (M0, M1, P, NX): S x n bits each.
int64_t query_bytes(const rpq_server *s, const Automaton &a) {
    const int64_t n = s->g->n, W = (n + 63) / 64;
    if (s->engine == 0) {
        int64_t S = 4;
        while (S < a.S) S *= 2;
        return 4 * S * W * 8 + S * n * 4;
    }
    return 4 * (int64_t)a.S * ((n + 7) / 8);
}

bool fits_budget(const rpq_server *s, int64_t bytes) {
    return s->budget <= 0 || s->inflight_bytes + bytes <= s->budget;
}

// caller holds s->mu
void admit_account(rpq_server *s, int64_t bytes) {
    s->inflight_bytes += bytes;
    s->inflight_n++;
    s->peak_bytes = std::max(s->peak_bytes, s->inflight_bytes);
    s->peak_inflight = std::max(s->peak_inflight, s->inflight_n);
    s->admitted++;
}

void retire_account(rpq_server *s, int64_t bytes) {
    s->inflight_bytes -= bytes;
    s->inflight_n--;
}

void lane_masks(const rpq_server *s, uint64_t active[kLW]) {
    for (int w = 0; w < kLW; w++) active[w] = 0;
    for (int i = 0; i < kLanes; i++)
        if (s->lane[i].busy && !s->lane[i].finished) active[i / 64] |= 1ull << (i % 64);
}

// Rebuilds the lane tables from the current lane -> automaton assignment and
// uploads them (stream-ordered before the next step).
rpq_status upload_tables(rpq_server *s) {
    std::vector<const Automaton *> autos(kLanes, nullptr);
    for (int i = 0; i < kLanes; i++)
        if (s->lane[i].busy) autos[i] = &s->lane[i].a;
    std::vector<LDir> dirs;
    std::vector<LUnit> units;
    std::vector<LSrc> srcs;
    std::vector<uint64_t> fmask, smask;
    rpq_status st = lane_build_tables(s->g, autos.data(), kLanes, s->K, &dirs, &units, &srcs, &fmask,
                                      &smask);
    if (st != RPQ_OK) return st;
    fmask.resize((size_t)s->ws->K * kLW, 0);
    LaneDyn dyn{};
    dyn.n_dirs = (int32_t)dirs.size();
    lane_masks(s, dyn.active);
    const size_t need_dirs = sizeof(LDir) * dirs.size(), need_units = sizeof(LUnit) * units.size(),
                 need_srcs = sizeof(LSrc) * srcs.size();
    if (need_dirs > s->o_units - s->o_dirs || need_units > s->o_srcs - s->o_units ||
        need_srcs > s->o_fm - s->o_srcs)
        return fail(RPQ_ERR_INVALID, "lane tables exceed the server's table space");
    uint8_t *hs = static_cast<uint8_t *>(s->staging);
    memcpy(hs + s->o_dyn, &dyn, sizeof(dyn));
    if (need_dirs) memcpy(hs + s->o_dirs, dirs.data(), need_dirs);
    if (need_units) memcpy(hs + s->o_units, units.data(), need_units);
    if (need_srcs) memcpy(hs + s->o_srcs, srcs.data(), need_srcs);
    memcpy(hs + s->o_fm, fmask.data(), sizeof(uint64_t) * fmask.size());
    uint8_t *dt = s->tables.as<uint8_t>();
    auto up = [&](size_t at, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dt + at, hs + at, bytes, cudaMemcpyHostToDevice, s->st)
                     : cudaSuccess;
    };
    RPQ_CUDA_TRY(up(s->o_dyn, sizeof(dyn)));
    RPQ_CUDA_TRY(up(s->o_dirs, need_dirs));
    RPQ_CUDA_TRY(up(s->o_units, need_units));
    RPQ_CUDA_TRY(up(s->o_srcs, need_srcs));
    RPQ_CUDA_TRY(up(s->o_fm, sizeof(uint64_t) * fmask.size()));
    return RPQ_OK;
}

void finish_ticket(rpq_server *s, uint64_t ticket, rpq_status status, std::vector<int32_t> ans,
                   Clock::time_point t_submit) {
    // caller holds s->mu
    Done d;
    d.status = status;
    d.answer = std::move(ans);
    s->results[ticket] = std::move(d);
    s->inflight.erase(ticket);
    s->completed++;
    const auto now = Clock::now();
    s->t_last = now;
    s->latency_ms.push_back(std::chrono::duration<double, std::milli>(now - t_submit).count());
}

void worker_main(rpq_server *s) {
    cudaSetDevice(s->g->device);
    int step = 0;
    bool tables_dirty = true;
    for (;;) {
        std::vector<int> admitted;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            auto busy = [&] {
                for (int i = 0; i < s->lanes_max; i++)
                    if (s->lane[i].busy) return true;
                return false;
            };
            // (a queued query that does not fit the budget waits for a lane
            // to retire, and some lane is then busy)
            s->cv.wait(lk, [&] { return s->stop || !s->queue.empty() || busy(); });
            if (s->stop) return;
            // admission: free lanes take queued queries, in order, while
            // their state fits the memory budget
            for (int i = 0; i < s->lanes_max && !s->queue.empty(); i++) {
                if (s->lane[i].busy) continue;
                if (s->queue.front().a.start_mask == 0) {  // empty language: empty answer
                    Pending q = std::move(s->queue.front());
                    s->queue.pop_front();
                    finish_ticket(s, q.ticket, RPQ_OK, {}, q.t_submit);
                    s->cv_done.notify_all();
                    i--;
                    continue;
                }
                const int64_t need = query_bytes(s, s->queue.front().a);
                if (!fits_budget(s, need)) break;
                Pending q = std::move(s->queue.front());
                s->queue.pop_front();
                Lane &L = s->lane[i];
                L.busy = true;
                L.finished = false;
                L.bytes = need;
                L.ticket = q.ticket;
                L.a = std::move(q.a);
                L.source = q.source;
                L.level = 0;
                L.t_submit = q.t_submit;
                admitted.push_back(i);
                admit_account(s, need);
            }
        }
        rpq_status err = RPQ_OK;
        if (!admitted.empty()) tables_dirty = true;
        if (tables_dirty) {
            err = upload_tables(s);
            tables_dirty = false;
        }
        // seeds of the admitted lanes into the current frontier
        if (err == RPQ_OK && !admitted.empty()) {
            std::map<std::tuple<int, int, int>, uint64_t> seedm;
            std::vector<int32_t> verts;
            for (int i : admitted) {
                const Lane &L = s->lane[i];
                for (int q = 0; q < L.a.S; q++)
                    if ((L.a.start_mask >> q) & 1)
                        seedm[std::make_tuple(L.source, q, i / 64)] |= 1ull << (i % 64);
                verts.push_back(L.source);
            }
            std::sort(verts.begin(), verts.end());
            verts.erase(std::unique(verts.begin(), verts.end()), verts.end());
            std::vector<int32_t> rec;
            for (auto &kv : seedm) {
                rec.push_back(std::get<0>(kv.first));
                rec.push_back(std::get<1>(kv.first));
                rec.push_back(std::get<2>(kv.first));
                rec.push_back((int32_t)(uint32_t)kv.second);
                rec.push_back((int32_t)(uint32_t)(kv.second >> 32));
            }
            uint8_t *hs = static_cast<uint8_t *>(s->staging);
            memcpy(hs + s->o_seed, rec.data(), sizeof(int32_t) * rec.size());
            memcpy(hs + s->o_verts, verts.data(), sizeof(int32_t) * verts.size());
            cudaError_t e = cudaMemcpyAsync(s->tables.as<uint8_t>() + s->o_seed, hs + s->o_seed,
                                            sizeof(int32_t) * rec.size(), cudaMemcpyHostToDevice,
                                            s->st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(s->tables.as<uint8_t>() + s->o_verts, hs + s->o_verts,
                                    sizeof(int32_t) * verts.size(), cudaMemcpyHostToDevice, s->st);
            if (e != cudaSuccess) err = fail(RPQ_ERR_CUDA, "seed upload: %s", cudaGetErrorString(e));
            if (err == RPQ_OK)
                err = lane_seed(s->p, reinterpret_cast<const int32_t *>(s->tables.as<uint8_t>() + s->o_seed),
                                (int)(rec.size() / 5),
                                reinterpret_cast<const int32_t *>(s->tables.as<uint8_t>() + s->o_verts),
                                (int)verts.size(), step, s->st);
        }
        // one level step for every lane
        if (err == RPQ_OK) {
            cudaError_t e = cudaGraphLaunch(s->step_exec, s->st);
            if (e == cudaSuccess) {
                g_kernel_launches.fetch_add(kLaneStepKernels, std::memory_order_relaxed);
                e = cudaMemcpyAsync(s->out_host, s->step_out.p, sizeof(LaneStepOut),
                                    cudaMemcpyDeviceToHost, s->st);
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
            if (e != cudaSuccess) err = fail(RPQ_ERR_CUDA, "level step: %s", cudaGetErrorString(e));
            else if (s->out_host->status != 0) err = (rpq_status)s->out_host->status;
        }
        // lanes whose frontier emptied (or that reached the level cap) stop
        // expanding at once; their answers are extracted in batches, so the
        // extract-and-clear pass over the visited set is shared
        if (err == RPQ_OK) {
            step = s->out_host->step;
            std::lock_guard<std::mutex> lk(s->mu);
            s->level_steps++;
            for (int i = 0; i < s->lanes_max; i++) {
                Lane &L = s->lane[i];
                if (!L.busy || L.finished) continue;
                L.level++;
                const bool grew = (s->out_host->lane_new[i / 64] >> (i % 64)) & 1ull;
                if (!grew || (s->max_levels > 0 && L.level >= s->max_levels)) {
                    L.finished = true;
                    L.finished_step = s->level_steps;
                    tables_dirty = true;  // drop the lane from the active mask
                }
            }
        }
        std::vector<int32_t> done_ids;
        if (err == RPQ_OK) {
            std::lock_guard<std::mutex> lk(s->mu);
            int running = 0, free_lanes = 0;
            int64_t oldest = -1;
            for (int i = 0; i < s->lanes_max; i++) {
                const Lane &L = s->lane[i];
                if (!L.busy) {
                    free_lanes++;
                } else if (L.finished) {
                    done_ids.push_back(i);
                    if (oldest < 0 || L.finished_step < oldest) oldest = L.finished_step;
                } else {
                    running++;
                }
            }
            const bool harvest = !done_ids.empty() &&
                                 ((int)done_ids.size() >= 16 || running == 0 ||
                                  (!s->queue.empty() && free_lanes == 0) ||
                                  s->level_steps - oldest >= 4);
            if (!harvest) done_ids.clear();
        }
        if (err == RPQ_OK && !done_ids.empty()) {
            std::vector<int64_t> offs;
            std::vector<int32_t> ans;
            err = lane_harvest(s->g, s->ws.get(), s->p,
                               reinterpret_cast<const uint64_t *>(s->tables.as<uint8_t>() + s->o_fm),
                               done_ids.data(), (int)done_ids.size(), &offs, &ans, s->st);
            if (err == RPQ_OK) {
                std::lock_guard<std::mutex> lk(s->mu);
                for (size_t k = 0; k < done_ids.size(); k++) {
                    Lane &L = s->lane[done_ids[k]];
                    std::vector<int32_t> a(ans.begin() + offs[k], ans.begin() + offs[k + 1]);
                    finish_ticket(s, L.ticket, RPQ_OK, std::move(a), L.t_submit);
                    retire_account(s, L.bytes);
                    L.busy = false;
                    L.finished = false;
                }
                tables_dirty = true;
            }
            s->cv_done.notify_all();
        }
        if (err != RPQ_OK) {
            // fail every query in flight; the server stops serving
            std::lock_guard<std::mutex> lk(s->mu);
            s->fatal = err;
            for (int i = 0; i < s->lanes_max; i++)
                if (s->lane[i].busy) {
                    finish_ticket(s, s->lane[i].ticket, err, {}, s->lane[i].t_submit);
                    retire_account(s, s->lane[i].bytes);
                    s->lane[i].busy = false;
                }
            while (!s->queue.empty()) {
                finish_ticket(s, s->queue.front().ticket, err, {}, s->queue.front().t_submit);
                s->queue.pop_front();
            }
            s->cv_done.notify_all();
            return;
        }
    }
}

// Query slots of a server on engine 0 by default: at 2,000 q/s on rmat20, 4,
// 6, 8 and 12 slots gave the same latencies (p50 0.15-0.16 ms, p99 1.16-1.17
// ms) and 9.7K, 11.5K, 12.7K and 11.1K q/s at saturation.
constexpr int kServeSlots = 8;

// Engine 0: one admitted query at a time per worker, on its own stream.  A
// query is admitted when a worker is free and its workspace fits the memory
// budget beside those of the queries in flight (in arrival order: a query
// that does not fit waits, and so do the ones behind it).  Its share of the
// persistent grid follows the queue at admission: 1/k of the grid when it
// and k - 1 queued queries are waiting (at most 1/slots), so a burst
// overlaps on the device, while a query that finds the queue empty takes
// half the grid (RPQ_SERVE_IDLE_DIV), so that one arriving meanwhile finds
// room beside it.  (A query admitted while others fill the grid waits for
// room either way: a cooperative launch starts only when all its CTAs fit.)
void slot_worker_main(rpq_server *s) {
    cudaSetDevice(s->g->device);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->fatal = RPQ_ERR_CUDA;
        return;
    }
    for (;;) {
        Pending q;
        int64_t need = 0;
        int grid_div = s->lanes_max;
        int alone_at_admit = 0;              // no other query in flight when admitted
        int64_t completed_at_admit = 0;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] {
                return s->stop ||
                       (!s->queue.empty() && s->inflight_n < s->slot_cap &&
                        fits_budget(s, query_bytes(s, s->queue.front().a)));
            });
            if (s->stop) break;
            q = std::move(s->queue.front());
            s->queue.pop_front();
            need = query_bytes(s, q.a);
            admit_account(s, need);
            alone_at_admit = s->inflight_n == 1;
            completed_at_admit = s->completed;
            grid_div = std::min(s->lanes_max, std::max(s->idle_div, 1 + (int)s->queue.size()));
        }
        int64_t cnt = 0;
        rpq_stats qs{};
        // the answer stays in this thread's pinned host buffer (the kernel
        // writes small ones there directly) and is copied once, into the
        // ticket's result
        const rpq_status r = run_query_slot(s->g, q.a, q.source, s->max_levels, nullptr, 0,
                                            nullptr, nullptr, &qs, &cnt, st, grid_div, true);
        rpq_status r_ans = r;
        std::vector<int32_t> ans;
        if (r == RPQ_OK && cnt > 0) {
            const int32_t *h = nullptr;
            int64_t hc = 0;
            if (last_host_answer(&h, &hc) == RPQ_OK && hc == cnt) ans.assign(h, h + hc);
            else r_ans = RPQ_ERR_CUDA;  // the answer did not reach the host buffer
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            // another query held device memory during this attempt if one was
            // in flight when it was admitted, still is, or ended meanwhile
            const bool shared =
                !alone_at_admit || s->inflight_n > 1 || s->completed != completed_at_admit;
            if (r == RPQ_ERR_OOM && shared) {
                // device memory ran out beside the other queries in flight:
                // admit fewer at once and run this query again when one ends
                retire_account(s, need);
                s->admitted--;
                s->slot_cap = std::max(1, s->inflight_n);
                s->oom_retries++;
                s->queue.push_front(std::move(q));
                s->cv.notify_all();
                continue;
            }
            finish_ticket(s, q.ticket, r_ans, std::move(ans), q.t_submit);
            retire_account(s, need);
            if (r == RPQ_OK && s->slot_cap < s->lanes_max && s->completed % 16 == 0)
                s->slot_cap++;
            // the levels this query expanded: its non-empty levels after
            // level 0, plus level 0 (the last expansion finds nothing)
            if (r == RPQ_OK) s->level_steps += qs.levels + 1;
        }
        s->cv.notify_all();  // a query waiting for memory may fit now
        s->cv_done.notify_all();
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
}

}  // namespace
}  // namespace rpq

using namespace rpq;

extern "C" rpq_status rpq_serve_create(const rpq_graph *g, const rpq_serve_config *cfg,
                                       rpq_server **out) {
    clear_error();
    if (!g || !out) return fail(RPQ_ERR_INVALID, "null argument");
    *out = nullptr;
    rpq_serve_config c{};
    if (cfg) c = *cfg;
    if (c.engine != 0 && c.engine != 1) return fail(RPQ_ERR_INVALID, "engine must be 0 or 1");
    if (c.engine == 0) {
        const int slots = c.max_lanes ? c.max_lanes : kServeSlots;
        if (slots <= 0 || slots > 64) return fail(RPQ_ERR_INVALID, "max_lanes (slots) must be in [1, 64]");
        if (c.max_levels < 0) return fail(RPQ_ERR_INVALID, "max_levels must be >= 0");
        std::unique_ptr<rpq_server> s(new rpq_server());
        s->g = const_cast<rpq_graph *>(g);
        s->engine = 0;
        s->lanes_max = slots;
        s->K = kMaxStates;
        s->max_levels = c.max_levels;
        s->queue_cap = c.queue_capacity > 0 ? (size_t)c.queue_capacity : 65536;
        s->budget = c.memory_budget;
        s->slot_cap = slots;
        const char *idv = getenv("RPQ_SERVE_IDLE_DIV");
        s->idle_div = std::max(1, std::min(slots, idv ? atoi(idv) : 2));
        rpq_server *raw = s.get();
        for (int k = 0; k < slots; k++) s->slot_workers.emplace_back(slot_worker_main, raw);
        *out = s.release();
        return RPQ_OK;
    }
    const int lanes = c.max_lanes ? c.max_lanes : kLanes;
    if (lanes <= 0 || lanes > kLanes) return fail(RPQ_ERR_INVALID, "max_lanes must be in [1, %d]", kLanes);
    const int K = c.max_states ? c.max_states : 16;
    if (K <= 0 || K > kLaneMaxSlots) return fail(RPQ_ERR_INVALID, "max_states must be in [1, %d]", kLaneMaxSlots);
    if (c.max_levels < 0) return fail(RPQ_ERR_INVALID, "max_levels must be >= 0");
    std::unique_ptr<rpq_server> s(new rpq_server());
    s->g = const_cast<rpq_graph *>(g);
    s->lanes_max = lanes;
    s->engine = 1;
    s->max_levels = c.max_levels;
    s->queue_cap = c.queue_capacity > 0 ? (size_t)c.queue_capacity : 65536;
    RPQ_CUDA_TRY(cudaSetDevice(g->device));
    // the lane arrays are allocated whole (max_states slots of max_lanes
    // lanes); the budget bounds the lane bits the admitted queries occupy
    s->budget = c.memory_budget;
    rpq_status st = lane_ws_acquire_fixed(s->g, K, &s->ws);
    if (st != RPQ_OK) return st;
    s->K = s->ws->K;
    // table space: dyn | dirs | units | srcs | fmask | seeds | seed vertices
    s->o_dyn = 0;
    s->o_dirs = 256;
    s->o_units = s->o_dirs + (64u << 10);
    s->o_srcs = s->o_units + (512u << 10);
    s->o_fm = s->o_srcs + (2u << 20);
    s->o_seed = s->o_fm + (size_t)kLaneMaxSlots * kLW * 8;
    s->o_verts = s->o_seed + (size_t)kLanes * kLaneMaxSlots * 5 * 4;
    if (s->o_verts + kLanes * 4 > kServeTablesBytes) return fail(RPQ_ERR_INVALID, "table layout");
    if (!s->tables.alloc(kServeTablesBytes) || !s->step_out.alloc(sizeof(LaneStepOut)))
        return fail(RPQ_ERR_OOM, "server buffers");
    RPQ_CUDA_TRY(cudaMallocHost(&s->staging, kServeTablesBytes));
    RPQ_CUDA_TRY(cudaMallocHost((void **)&s->out_host, sizeof(LaneStepOut)));
    memset(s->staging, 0, kServeTablesBytes);
    RPQ_CUDA_TRY(cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking));
    // clean lane state
    const size_t words = (size_t)g->n * s->K * kLW;
    RPQ_CUDA_TRY(cudaMemsetAsync(s->ws->P.p, 0, words * 8, s->st));
    RPQ_CUDA_TRY(cudaMemsetAsync(s->ws->M0.p, 0, words * 8, s->st));
    RPQ_CUDA_TRY(cudaMemsetAsync(s->ws->M1.p, 0, words * 8, s->st));
    RPQ_CUDA_TRY(cudaMemsetAsync(s->ws->ctr.p, 0, sizeof(LaneCounters), s->st));
    RPQ_CUDA_TRY(cudaMemsetAsync(s->tables.p, 0, kServeTablesBytes, s->st));
    s->p = lane_params(s->g, s->ws.get(), 0, 0, 0, 0);
    uint8_t *dt = s->tables.as<uint8_t>();
    s->p.dyn = reinterpret_cast<const LaneDyn *>(dt + s->o_dyn);
    s->p.dirs = reinterpret_cast<const LDir *>(dt + s->o_dirs);
    s->p.units = reinterpret_cast<const LUnit *>(dt + s->o_units);
    s->p.srcs = reinterpret_cast<const LSrc *>(dt + s->o_srcs);
    st = lane_capture_step(s->p, s->step_out.as<LaneStepOut>(), s->st, &s->step_exec);
    if (st != RPQ_OK) return st;
    RPQ_CUDA_TRY(cudaStreamSynchronize(s->st));
    rpq_server *raw = s.get();
    s->worker = std::thread(worker_main, raw);
    *out = s.release();
    return RPQ_OK;
}

extern "C" rpq_status rpq_serve_submit(rpq_server *s, const rpq_nfa *nfa, int32_t source,
                                       uint64_t *ticket) {
    clear_error();
    if (!s || !nfa || !ticket) return fail(RPQ_ERR_INVALID, "null argument");
    const Automaton &a = nfa->a;
    if (source < 0 || source >= s->g->n)
        return fail(RPQ_ERR_INVALID, "source %d outside [0, %d)", source, s->g->n);
    if (a.S > s->K) return fail(RPQ_ERR_INVALID, "automaton has %d states; the server holds %d", a.S, s->K);
    for (size_t t = 0; t < a.sym.size(); t++) {
        const int lab = a.sym[t] < a.L ? a.sym[t] : a.sym[t] - a.L;
        if (lab >= s->g->L) return fail(RPQ_ERR_INVALID, "label %d is not a label of the graph", lab);
    }
    if (s->budget > 0 && query_bytes(s, a) > s->budget)
        return fail(RPQ_ERR_OOM, "the query needs %lld bytes of device state, budget %lld",
                    (long long)query_bytes(s, a), (long long)s->budget);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal != RPQ_OK) return fail(s->fatal, "server stopped after a device error");
    if (s->queue.size() >= s->queue_cap) {
        s->rejected++;
        return fail(RPQ_ERR_BUSY, "queue full");
    }
    Pending q;
    q.ticket = s->next_ticket++;
    q.a = a;
    q.source = source;
    q.t_submit = Clock::now();
    if (!s->started) {
        s->started = true;
        s->t_first = q.t_submit;
    }
    *ticket = q.ticket;
    s->inflight[q.ticket] = 1;
    s->queue.push_back(std::move(q));
    s->submitted++;
    s->cv.notify_one();
    return RPQ_OK;
}

extern "C" rpq_status rpq_serve_poll(rpq_server *s, uint64_t ticket, int32_t *out_vertices,
                                     int64_t capacity, int64_t *out_count) {
    clear_error();
    if (!s || !out_count || capacity < 0 || (capacity > 0 && !out_vertices))
        return fail(RPQ_ERR_INVALID, "bad argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) {
        if (s->inflight.count(ticket)) return RPQ_ERR_BUSY;
        return fail(RPQ_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    }
    if (it->second.status != RPQ_OK) {
        const rpq_status e = it->second.status;
        s->results.erase(it);
        return fail(e, "query failed on the device");
    }
    const int64_t n = (int64_t)it->second.answer.size();
    *out_count = n;
    if (n > capacity) return fail(RPQ_ERR_CAPACITY, "answer has %lld vertices", (long long)n);
    if (n) {
        if (is_device_pointer(out_vertices)) {
            if (cudaMemcpy(out_vertices, it->second.answer.data(), 4 * n, cudaMemcpyHostToDevice) !=
                cudaSuccess)
                return fail(RPQ_ERR_CUDA, "copy to device output");
        } else {
            memcpy(out_vertices, it->second.answer.data(), 4 * n);
        }
    }
    s->results.erase(it);
    return RPQ_OK;
}

extern "C" rpq_status rpq_serve_drain(rpq_server *s, int64_t timeout_ms) {
    clear_error();
    if (!s) return fail(RPQ_ERR_INVALID, "null argument");
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                        [&] { return s->inflight.empty(); });
    if (!ok) return fail(RPQ_ERR_TIMEOUT, "%zu queries still in flight", s->inflight.size());
    return RPQ_OK;
}

extern "C" rpq_status rpq_serve_stats_get(rpq_server *s, struct rpq_serve_stats *out) {
    clear_error();
    if (!s || !out) return fail(RPQ_ERR_INVALID, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    rpq_serve_stats_t r{};
    r.submitted = s->submitted;
    r.admitted = s->admitted;
    r.completed = s->completed;
    r.rejected = s->rejected;
    r.level_steps = s->level_steps;
    r.peak_in_flight = s->peak_inflight;
    r.peak_bytes = s->peak_bytes;
    r.oom_retries = s->oom_retries;
    if (!s->latency_ms.empty()) {
        std::vector<double> v = s->latency_ms;
        std::sort(v.begin(), v.end());
        r.p50_ms = v[v.size() / 2];
        r.p99_ms = v[std::min(v.size() - 1, (size_t)(0.99 * (double)v.size()))];
        double sum = 0;
        for (double x : v) sum += x;
        r.mean_ms = sum / (double)v.size();
    }
    if (s->started && s->completed > 0) {
        r.elapsed_s = std::chrono::duration<double>(s->t_last - s->t_first).count();
        r.qps = r.elapsed_s > 0 ? (double)s->completed / r.elapsed_s : 0.0;
    }
    *out = r;
    return RPQ_OK;
}

extern "C" rpq_status rpq_serve_stats(rpq_server *s, struct rpq_serve_stats *out) {
    return rpq_serve_stats_get(s, out);
}

extern "C" void rpq_serve_destroy(rpq_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto &t : s->slot_workers)
        if (t.joinable()) t.join();
    if (s->st) cudaStreamSynchronize(s->st);
    if (s->step_exec) cudaGraphExecDestroy(s->step_exec);
    if (s->staging) cudaFreeHost(s->staging);
    if (s->out_host) cudaFreeHost(s->out_host);
    if (s->ws) {
        // leave the workspace clean for the next user
        const size_t words = (size_t)s->g->n * s->ws->K * kLW;
        cudaMemsetAsync(s->ws->P.p, 0, words * 8, s->st);
        cudaMemsetAsync(s->ws->M0.p, 0, words * 8, s->st);
        cudaMemsetAsync(s->ws->M1.p, 0, words * 8, s->st);
        cudaMemsetAsync(s->ws->ctr.p, 0, sizeof(LaneCounters), s->st);
        cudaStreamSynchronize(s->st);
        lane_ws_return(s->g, std::move(s->ws));
    }
    if (s->st) cudaStreamDestroy(s->st);
    delete s;
}
