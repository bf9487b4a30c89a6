// cm_server.cu -- request loop that keeps graphs resident on the GPU and
// serves update batches to them (host code; the maintenance itself is the
// ordinary update path of cm_capi.cu and its captured steps).
//
// Per resident graph the server runs two threads:
//   copier  admits queued requests in arrival order while the graph's slice
//           of the device-memory budget has room: it reserves a contiguous
//           range of the graph's insert or delete arena (two rings) and
//           copies the batch there on its own stream, so admission overlaps
//           the maintenance call that is running;
//   worker  takes the oldest admitted requests as one round: the longest
//           run in arrival order whose inserted edges and deleted edges are
//           disjoint (so applying all of its inserts and then all of its
//           deletes is what applying the requests one by one does) and that
//           is contiguous in both rings, up to max_round edges.  A round is
//           ONE captured update step (cm_step: the insert batch, then the
//           delete batch, Algorithms 1 and 5, one CUDA graph replay), or a
//           plain call when it holds one kind of request only.  It records
//           the round's result for each request and frees the arena ranges.
// Graphs are served by independent threads on their own streams, so their
// calls overlap on the device.  A round only reorders requests whose edge
// sets do not meet, so every graph ends in the state of applying its
// requests one by one (its cores are a function of its edge set,
// Definitions 1-2), whatever the arrival timing or the other graphs'
// traffic.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/coremaint.h"

namespace {

using Clock = std::chrono::steady_clock;

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

struct Req {
    int64_t id = 0;
    int32_t graph = 0, op = 0;
    int64_t k = 0;
    std::vector<int32_t> edges;   // host copy until admitted
    std::vector<uint64_t> keys;   // canonical edge keys, for the round's disjointness test
    int64_t t_submit = 0, t_admit = 0, t_done = 0;
    int64_t off = 0;              // arena position (pairs, monotone; slot = off % cap)
    int64_t round = -1, round_applied = 0, round_edges = 0, round_requests = 0;
    int32_t status = 0;
    bool done = false;
};

struct Ring {                      // staged batches of one operation
    int32_t* arena = nullptr;
    int64_t cap = 0;               // pairs
    int64_t tail = 0;              // next free position (monotone)
    std::deque<Req*> resident;     // holding arena space, in allocation order
};

struct Slot {
    cm_graph* h = nullptr;
    cm_step* step = nullptr;       // insert + delete rounds as one replay (NULL: plain calls)
    cudaStream_t copy_stream = nullptr;
    Ring ring[2];                  // 0 inserts, 1 deletes
    std::deque<Req*> queued;       // submitted, not admitted
    std::deque<Req*> admitted;     // copied, waiting for a round
    std::thread copier, worker;
    std::condition_variable cv_copy, cv_work;
    std::mutex graph_mu;           // held during a call on h
    int64_t rounds = 0;
};

}  // namespace

struct cm_server {
    std::vector<Slot*> slots;
    int64_t max_round = 0;
    std::mutex mu;
    std::condition_variable cv_done;
    std::unordered_map<int64_t, Req*> reqs;
    int64_t next_id = 1;
    bool stop = false;
    int64_t submitted = 0, completed = 0, rounds = 0, coalesced = 0, failed = 0;
    int64_t edges_done = 0;
};

namespace {

// Arena position for k pairs, or -1 if the ring has no contiguous room now.
int64_t arena_reserve(Ring& s, int64_t k) {
    int64_t at = s.tail;
    const int64_t in_slot = at % s.cap;
    if (in_slot + k > s.cap) at += s.cap - in_slot;   // would wrap: start at the ring's beginning
    const int64_t head = s.resident.empty() ? at : s.resident.front()->off;
    if (at + k - head > s.cap) return -1;
    return at;
}

inline uint64_t canon(int32_t a, int32_t b) {
    const uint32_t lo = (uint32_t)(a < b ? a : b), hi = (uint32_t)(a < b ? b : a);
    return ((uint64_t)lo << 32) | hi;
}

void copier_loop(cm_server* S, Slot* s) {
    for (;;) {
        Req* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            s->cv_copy.wait(lk, [&] {
                return S->stop || (!s->queued.empty() &&
                                   arena_reserve(s->ring[s->queued.front()->op], s->queued.front()->k) >= 0);
            });
            if (S->stop) return;
            r = s->queued.front();
            s->queued.pop_front();
            Ring& g = s->ring[r->op];
            r->off = arena_reserve(g, r->k);
            g.tail = r->off + r->k;
            g.resident.push_back(r);
        }
        Ring& g = s->ring[r->op];
        cudaError_t e = cudaMemcpyAsync(g.arena + 2 * (r->off % g.cap), r->edges.data(), (size_t)r->k * 8,
                                        cudaMemcpyHostToDevice, s->copy_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy_stream);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            r->t_admit = now_ns();
            if (e != cudaSuccess) r->status = CM_ERR_CUDA;
            std::vector<int32_t>().swap(r->edges);
            s->admitted.push_back(r);
        }
        s->cv_work.notify_one();
    }
}

int run_call(cm_graph* h, int op, const int32_t* E, int64_t k, int64_t* applied) {
    return op == CM_OP_INSERT ? cm_insert_edges(h, E, k, applied) : cm_delete_edges(h, E, k, applied);
}

void worker_loop(cm_server* S, Slot* s) {
    std::unordered_set<uint64_t> seen[2];
    for (;;) {
        std::vector<Req*> round;
        int64_t total[2] = {0, 0};
        {
            std::unique_lock<std::mutex> lk(S->mu);
            s->cv_work.wait(lk, [&] { return S->stop || !s->admitted.empty(); });
            if (S->stop) return;
            // the longest run of admitted requests whose inserted and deleted
            // edges are disjoint, contiguous in both rings, within max_round
            seen[0].clear();
            seen[1].clear();
            int64_t end[2] = {-1, -1};
            while (!s->admitted.empty()) {
                Req* r = s->admitted.front();
                if (r->status != 0) {
                    if (round.empty()) {   // a failed copy: report it alone
                        round.push_back(r);
                        s->admitted.pop_front();
                    }
                    break;
                }
                const int op = r->op, other = 1 - r->op;
                if ((end[op] >= 0 && r->off != end[op]) || (!round.empty() && total[0] + total[1] + r->k > S->max_round))
                    break;
                bool meets = false;
                for (uint64_t k : r->keys)
                    if (seen[other].count(k)) { meets = true; break; }
                if (meets) break;
                for (uint64_t k : r->keys) seen[op].insert(k);
                round.push_back(r);
                total[op] += r->k;
                end[op] = r->off + r->k;
                s->admitted.pop_front();
            }
        }
        // outcome per operation: the step (or the pair of plain calls)
        int op_rc[2] = {round.front()->status, round.front()->status};
        int64_t op_applied[2] = {0, 0};
        std::vector<int> alone_rc(round.size(), 0);   // per request, after a rejected call
        std::vector<int64_t> alone_applied(round.size(), 0);
        std::vector<char> solo(round.size(), 0);
        if (op_rc[0] == 0) {
            std::lock_guard<std::mutex> g(s->graph_mu);
            const int32_t* E[2] = {nullptr, nullptr};
            for (Req* r : round)
                if (!E[r->op]) E[r->op] = s->ring[r->op].arena + 2 * (r->off % s->ring[r->op].cap);
            if (total[0] > 0 && total[1] > 0 && s->step) {
                const int rc = cm_step_run(s->step, &total[0], E[0], &total[1], E[1], &op_applied[0], &op_applied[1]);
                op_rc[0] = op_rc[1] = rc;
            } else {
                for (int op = 0; op < 2; op++)
                    op_rc[op] = total[op] > 0 ? run_call(s->h, op, E[op], total[op], &op_applied[op]) : 0;
            }
            // a call validates its whole batch before changing anything, so a
            // rejected one applied nothing: replay its requests one by one, in
            // order, so that only the offending ones fail
            for (size_t i = 0; i < round.size(); i++) {
                Req* r = round[i];
                if (op_rc[r->op] != CM_ERR_INVALID || round.size() == 1) continue;
                const Ring& g = s->ring[r->op];
                solo[i] = 1;
                alone_rc[i] = run_call(s->h, r->op, g.arena + 2 * (r->off % g.cap), r->k, &alone_applied[i]);
            }
        }
        const int64_t t = now_ns();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            const int64_t rid = S->rounds;
            int64_t nsolo = 0;
            for (size_t i = 0; i < round.size(); i++) {
                Req* r = round[i];
                if (solo[i]) {
                    r->round = rid + 1 + nsolo++;
                    r->round_applied = alone_applied[i];
                    r->round_edges = r->k;
                    r->round_requests = 1;
                    r->status = alone_rc[i];
                } else {
                    r->round = rid;
                    r->round_applied = op_applied[0] + op_applied[1];
                    r->round_edges = total[0] + total[1];
                    r->round_requests = (int64_t)round.size();
                    r->status = op_rc[r->op];
                }
                r->t_done = t;
                r->done = true;
                std::vector<uint64_t>().swap(r->keys);
                if (r->status) S->failed++;
                else S->edges_done += r->k;
                // the round's requests are the oldest residents of their ring
                std::deque<Req*>& res = s->ring[r->op].resident;
                if (!res.empty() && res.front() == r) res.pop_front();
                else res.erase(std::find(res.begin(), res.end(), r));
            }
            S->rounds += 1 + nsolo;
            s->rounds += 1 + nsolo;
            S->completed += (int64_t)round.size();
            S->coalesced += (int64_t)round.size() - 1 - nsolo;
        }
        s->cv_copy.notify_one();
        S->cv_done.notify_all();
    }
}

int64_t percentile(std::vector<int64_t> v, double q) {
    if (v.empty()) return 0;
    std::sort(v.begin(), v.end());
    size_t i = (size_t)(q * (double)(v.size() - 1) + 0.5);
    return v[std::min(i, v.size() - 1)];
}

}  // namespace

extern "C" int cm_server_create(cm_server** out, cm_graph* const* graphs, int32_t ngraphs,
                                int64_t device_budget_bytes, int64_t max_round_edges) {
    if (!out || !graphs || ngraphs <= 0 || device_budget_bytes < 16 * ngraphs) return CM_ERR_INVALID;
    *out = nullptr;
    cm_server* S = new (std::nothrow) cm_server();
    if (!S) return CM_ERR_OOM;
    S->max_round = max_round_edges > 0 ? max_round_edges : (int64_t)1 << 40;
    const int64_t per = device_budget_bytes / ngraphs / 16;   // pairs per ring (two rings per graph)
    for (int32_t i = 0; i < ngraphs; i++) {
        Slot* s = new (std::nothrow) Slot();
        if (!s || !graphs[i]) {
            delete s;
            cm_server_destroy(S);
            return CM_ERR_INVALID;
        }
        S->slots.push_back(s);
        s->h = graphs[i];
        for (Ring& g : s->ring) g.cap = per;
        if (cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMalloc(&s->ring[0].arena, (size_t)per * 8) != cudaSuccess ||
            cudaMalloc(&s->ring[1].arena, (size_t)per * 8) != cudaSuccess) {
            cudaGetLastError();
            cm_server_destroy(S);
            return CM_ERR_OOM;
        }
        // mixed rounds run as one captured step where the handle allows it
        // (a created stream); otherwise as two plain calls
        const int64_t cap = per < S->max_round ? per : S->max_round;
        if (cm_step_create(&s->step, s->h, cap, cap, nullptr) != CM_OK) s->step = nullptr;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    for (Slot* s : S->slots) {
        s->copier = std::thread([S, s, dev] { cudaSetDevice(dev); copier_loop(S, s); });
        s->worker = std::thread([S, s, dev] { cudaSetDevice(dev); worker_loop(S, s); });
    }
    *out = S;
    return CM_OK;
}

extern "C" void cm_server_destroy(cm_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    for (Slot* s : S->slots) {
        s->cv_copy.notify_all();
        s->cv_work.notify_all();
    }
    S->cv_done.notify_all();
    for (Slot* s : S->slots) {
        if (s->copier.joinable()) s->copier.join();
        if (s->worker.joinable()) s->worker.join();
        if (s->step) cm_step_destroy(s->step);
        for (Ring& g : s->ring)
            if (g.arena) cudaFree(g.arena);
        if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
        delete s;
    }
    for (auto& kv : S->reqs) delete kv.second;
    delete S;
}

extern "C" int cm_server_submit(cm_server* S, int32_t graph, int32_t op, const int32_t* edges, int64_t k,
                                int64_t* request_id) {
    if (!S || graph < 0 || graph >= (int32_t)S->slots.size() || (op != CM_OP_INSERT && op != CM_OP_DELETE) ||
        k <= 0 || !edges)
        return CM_ERR_INVALID;
    Slot* s = S->slots[(size_t)graph];
    if (k > s->ring[op].cap) return CM_ERR_CAPACITY;   // can never be admitted
    Req* r = new (std::nothrow) Req();
    if (!r) return CM_ERR_OOM;
    r->graph = graph;
    r->op = op;
    r->k = k;
    r->edges.assign(edges, edges + 2 * k);
    r->keys.resize((size_t)k);
    for (int64_t i = 0; i < k; i++) r->keys[(size_t)i] = canon(edges[2 * i], edges[2 * i + 1]);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) {
            delete r;
            return CM_ERR_STATE;
        }
        r->id = S->next_id++;
        r->t_submit = now_ns();
        S->reqs[r->id] = r;
        s->queued.push_back(r);
        S->submitted++;
    }
    s->cv_copy.notify_one();
    if (request_id) *request_id = r->id;
    return CM_OK;
}

static void fill_result(const Req* r, cm_request_result* out) {
    out->status = r->status;
    out->round = r->round;
    out->round_applied = r->round_applied;
    out->round_edges = r->round_edges;
    out->round_requests = r->round_requests;
    out->latency_ns = r->t_done - r->t_submit;
    out->queue_ns = r->t_admit - r->t_submit;
}

extern "C" int cm_server_wait(cm_server* S, int64_t request_id, cm_request_result* out) {
    if (!S) return CM_ERR_INVALID;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(request_id);
    if (it == S->reqs.end()) return CM_ERR_INVALID;
    Req* r = it->second;
    S->cv_done.wait(lk, [&] { return r->done || S->stop; });
    if (!r->done) return CM_ERR_STATE;
    if (out) fill_result(r, out);
    return r->status;
}

extern "C" int cm_server_drain(cm_server* S) {
    if (!S) return CM_ERR_INVALID;
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_done.wait(lk, [&] { return S->completed == S->submitted || S->stop; });
    return S->failed ? CM_ERR_STATE : CM_OK;
}

extern "C" int cm_server_get_cores(cm_server* S, int32_t graph, int32_t* out) {
    if (!S || graph < 0 || graph >= (int32_t)S->slots.size()) return CM_ERR_INVALID;
    Slot* s = S->slots[(size_t)graph];
    std::lock_guard<std::mutex> g(s->graph_mu);
    return cm_get_cores(s->h, out, nullptr);
}

extern "C" int cm_server_get_stats(cm_server* S, cm_server_stats* out) {
    if (!S || !out) return CM_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->rounds = S->rounds;
    out->coalesced = S->coalesced;
    out->failed = S->failed;
    out->edges = S->edges_done;
    std::vector<int64_t> lat;
    for (auto& kv : S->reqs)
        if (kv.second->done) lat.push_back(kv.second->t_done - kv.second->t_submit);
    out->p50_ns = percentile(lat, 0.50);
    out->p99_ns = percentile(lat, 0.99);
    return CM_OK;
}

// Open-loop load: request i is submitted at start + arrival_ns[i] by a
// driver thread, whatever the state of earlier requests; its latency runs
// from that scheduled time to the end of its round.
extern "C" int cm_server_run_trace(cm_server* S, int64_t nreq, const int64_t* arrival_ns, const int32_t* graph,
                                   const int32_t* op, const int64_t* counts, const int32_t* edges,
                                   int64_t* latency_ns, int64_t* round_of, double* wall_s) {
    if (!S || nreq < 0 || (nreq > 0 && (!arrival_ns || !graph || !op || !counts || !edges))) return CM_ERR_INVALID;
    std::vector<int64_t> ids((size_t)nreq, 0), off((size_t)nreq + 1, 0);
    for (int64_t i = 0; i < nreq; i++) off[(size_t)i + 1] = off[(size_t)i] + counts[i];
    std::atomic<int> bad{0};
    const Clock::time_point t0 = Clock::now();
    std::thread driver([&] {
        for (int64_t i = 0; i < nreq; i++) {
            std::this_thread::sleep_until(t0 + std::chrono::nanoseconds(arrival_ns[i]));
            int rc = cm_server_submit(S, graph[i], op[i], edges + 2 * off[(size_t)i], counts[i], &ids[(size_t)i]);
            if (rc) bad.store(rc);
        }
    });
    driver.join();
    const int64_t start = std::chrono::duration_cast<std::chrono::nanoseconds>(t0.time_since_epoch()).count();
    int status = bad.load();
    int64_t last = start;
    for (int64_t i = 0; i < nreq && !status; i++) {
        cm_request_result r;
        int rc = cm_server_wait(S, ids[(size_t)i], &r);
        if (rc) {
            status = rc;
            break;
        }
        const Req* q;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            q = S->reqs[ids[(size_t)i]];
        }
        if (latency_ns) latency_ns[i] = q->t_done - (start + arrival_ns[i]);
        if (round_of) round_of[i] = q->round;
        last = std::max(last, q->t_done);
    }
    if (wall_s) *wall_s = (double)(last - start) * 1e-9;
    return status;
}
