// Query server with continuous batching over resident graphs.
//
// The paper runs one traversal at a time.  A server receives many traversal
// queries over a set of resident graphs; this one keeps every graph's CSR
// where it was loaded, keeps per-worker traversal buffers resident on the
// device, and admits work by a device-memory budget:
//   * queries are queued as they arrive (any thread may submit);
//   * whenever a worker slot is idle, the scheduler forms a job from the
//     oldest pending query: a BFS query takes every other pending BFS query of
//     the same graph with it, up to 64 and as many as the budget allows, and
//     runs them as one multi-source pass (one read of each list serves all of
//     them); an SSSP query runs alone;
//   * a job is admitted only when its device bytes (the worker's buffers for
//     that graph plus the batch's level rows) fit the budget; idle workers'
//     buffers are released first, and otherwise the job waits;
//   * each worker owns a CUDA stream (through its own share of each graph),
//     so jobs of different workers overlap on the GPU, and queries arriving
//     while others run join the next job: continuous batching.
// Results are the exact traversal outputs, identical alone or in a mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace emogi {
namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
    uint64_t ticket = 0;
    emogi_graph g = nullptr;
    uint32_t kind = 0;
    uint64_t src = 0;
    uint32_t* out = nullptr;
    Clock::time_point submitted, started, finished;
    emogi_query_result res{};
    bool done = false;
};

struct Job {
    emogi_graph g = nullptr;
    uint32_t kind = 0;
    std::vector<std::shared_ptr<Request>> reqs;
    uint64_t bytes = 0;  // device bytes admitted for this job
};

struct Slot {
    std::thread th;
    std::unique_ptr<Job> job;
    bool busy = false;
    std::unordered_map<emogi_graph, emogi_graph> views;  // graph -> this worker's share
    std::unordered_map<emogi_graph, uint64_t> view_bytes;
    uint32_t* dbuf = nullptr;  // level rows of a multi-source job
    size_t dbuf_bytes = 0;
};

// Device bytes a traversal handle's buffers take for a graph of n vertices
// and m edges (two frontier queues, the state array, SSSP stamps, far flags
// and last-expanded distances, the next-frontier flag bytes, the split-list
// queue, multi-source masks); mirrors the library's workspace layout.
uint64_t workspace_estimate(emogi_graph g) {
    const uint64_t n = g->n ? g->n : 1;
    const uint64_t lq = std::min<uint64_t>(n, g->m / 497 + 1);
    return 6 * 4 * n + (n / 16 + 1) * 16 + 20 * lq + 3 * 8 * n + 1024;
}

}  // namespace
}  // namespace emogi

struct emogi_server_s {
    emogi_server_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<std::shared_ptr<emogi::Request>> pending;
    std::unordered_map<uint64_t, std::shared_ptr<emogi::Request>> by_ticket;
    std::vector<std::unique_ptr<emogi::Slot>> slots;
    std::thread scheduler;
    uint64_t next_ticket = 1;
    uint64_t bytes_in_use = 0;
    uint64_t in_flight = 0;
    bool stopping = false;
};

using namespace emogi;

namespace {

void finish_request(emogi_server s, const std::shared_ptr<Request>& r, emogi_status st, uint32_t batch,
                    uint64_t reached, uint64_t scanned, Clock::time_point started) {
    r->finished = Clock::now();
    r->res.status = st;
    r->res.batch_size = batch;
    r->res.queue_ms = ms_between(r->submitted, started);
    r->res.run_ms = ms_between(started, r->finished);
    r->res.latency_ms = ms_between(r->submitted, r->finished);
    r->res.edges_reached = reached;
    r->res.edges_scanned = scanned;
    (void)s;
}

// Runs one job on a worker (no server lock held).
void run_job(emogi_server s, Slot& slot, Job& job) {
    const Clock::time_point t0 = Clock::now();
    emogi_status st = EMOGI_OK;
    std::string err;
    emogi_graph view = nullptr;
    {
        auto it = slot.views.find(job.g);
        if (it != slot.views.end()) {
            view = it->second;
        } else {
            st = emogi_graph_share(job.g, &view);
            if (st == EMOGI_OK) slot.views[job.g] = view;
        }
    }
    const uint64_t n = job.g->n;
    const uint32_t k = (uint32_t)job.reqs.size();
    std::vector<uint64_t> reached(k, 0), scanned(k, 0);
    emogi_opts o;
    memset(&o, 0, sizeof o);
    o.struct_size = sizeof o;
    if (st == EMOGI_OK && job.kind == EMOGI_QUERY_BFS && k > 1) {
        const size_t need = (size_t)k * n * 4;
        if (slot.dbuf_bytes < need) {
            if (slot.dbuf) dev_free(slot.dbuf, slot.dbuf_bytes);
            slot.dbuf = nullptr;
            slot.dbuf_bytes = 0;
            st = dev_alloc((void**)&slot.dbuf, need, "server level rows");
            if (st == EMOGI_OK) slot.dbuf_bytes = need;
        }
        if (st == EMOGI_OK) {
            std::vector<uint64_t> srcs(k);
            for (uint32_t i = 0; i < k; i++) srcs[i] = job.reqs[i]->src;
            o.out_on_device = 1;
            emogi_stats stt;
            st = emogi_msbfs(view, srcs.data(), k, slot.dbuf, &o, &stt);
            for (uint32_t i = 0; st == EMOGI_OK && i < k; i++) {
                if (!job.reqs[i]->out) continue;
                cudaError_t e = cudaMemcpyAsync(job.reqs[i]->out, slot.dbuf + (size_t)i * n, n * 4,
                                                cudaMemcpyDeviceToHost, view->stream);
                if (e != cudaSuccess) st = fail(EMOGI_E_CUDA, "result copy: %s", cudaGetErrorString(e));
            }
            if (st == EMOGI_OK && cudaStreamSynchronize(view->stream) != cudaSuccess)
                st = fail(EMOGI_E_CUDA, "result copy failed");
            // per-source reached edges are not split out by the pass; report the batch total
            for (uint32_t i = 0; i < k; i++) {
                reached[i] = stt.edges_reached / k;
                scanned[i] = stt.edges_scanned / k;
            }
        }
    } else if (st == EMOGI_OK) {
        for (uint32_t i = 0; i < k && st == EMOGI_OK; i++) {
            Request& r = *job.reqs[i];
            uint32_t* out = r.out;
            if (!out) {  // result not wanted: keep it on the device
                if (slot.dbuf_bytes < n * 4) {
                    if (slot.dbuf) dev_free(slot.dbuf, slot.dbuf_bytes);
                    slot.dbuf = nullptr;
                    slot.dbuf_bytes = 0;
                    st = dev_alloc((void**)&slot.dbuf, n * 4, "server level rows");
                    if (st != EMOGI_OK) break;
                    slot.dbuf_bytes = n * 4;
                }
                out = slot.dbuf;
                o.out_on_device = 1;
            } else {
                o.out_on_device = 0;
            }
            emogi_stats stt;
            st = job.kind == EMOGI_QUERY_SSSP ? emogi_sssp(view, r.src, out, &o, &stt)
                                              : emogi_bfs(view, r.src, out, &o, &stt);
            if (st == EMOGI_OK) {
                reached[i] = stt.edges_reached;
                scanned[i] = stt.edges_scanned;
            }
        }
    }
    if (st != EMOGI_OK) err = emogi_last_error();
    std::lock_guard<std::mutex> lk(s->mu);
    for (uint32_t i = 0; i < k; i++) {
        finish_request(s, job.reqs[i], st, k, reached[i], scanned[i], t0);
        job.reqs[i]->started = t0;
        job.reqs[i]->done = true;
    }
    if (st != EMOGI_OK) set_error(err);
}

void worker_main(emogi_server s, Slot* slot) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv_sched.wait(lk, [&] { return slot->job || (s->stopping && !slot->busy); });
        if (!slot->job) return;
        std::unique_ptr<Job> job = std::move(slot->job);
        lk.unlock();
        run_job(s, *slot, *job);
        lk.lock();
        s->bytes_in_use -= job->bytes;
        slot->busy = false;
        s->in_flight -= job->reqs.size();
        s->cv_done.notify_all();
        s->cv_sched.notify_all();
    }
}

uint64_t slot_bytes(const Slot& sl) {
    uint64_t b = sl.dbuf_bytes;
    for (auto& kv : sl.view_bytes) b += kv.second;
    return b;
}

// Releases a slot's resident buffers except its share of `keep` (caller holds
// the lock; the slot is idle, so nothing of it runs on the GPU).
void evict(emogi_server s, Slot& sl, emogi_graph keep) {
    for (auto it = sl.views.begin(); it != sl.views.end();) {
        if (it->first == keep) { ++it; continue; }
        s->bytes_in_use -= sl.view_bytes[it->first];
        sl.view_bytes.erase(it->first);
        emogi_free_graph(it->second);
        it = sl.views.erase(it);
    }
    if (sl.dbuf) {
        s->bytes_in_use -= sl.dbuf_bytes;
        dev_free(sl.dbuf, sl.dbuf_bytes);
        sl.dbuf = nullptr;
        sl.dbuf_bytes = 0;
    }
}

// Picks the next job and its worker; every device byte a worker holds (its
// graph shares' buffers and its level-row buffer) is charged to the budget
// while it lives.
void scheduler_main(emogi_server s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv_sched.wait(lk, [&] {
            if (s->stopping && s->pending.empty()) return true;
            if (s->pending.empty()) return false;
            for (auto& sp : s->slots)
                if (!sp->busy) return true;
            return false;
        });
        if (s->stopping && s->pending.empty()) return;
        auto head = s->pending.front();
        const emogi_graph g = head->g;
        const uint64_t n = g->n ? g->n : 1;
        // prefer an idle worker that already holds buffers for this graph
        Slot* slot = nullptr;
        for (auto& sp : s->slots)
            if (!sp->busy && sp->views.count(g)) { slot = sp.get(); break; }
        if (!slot)
            for (auto& sp : s->slots)
                if (!sp->busy) { slot = sp.get(); break; }
        const uint64_t B = s->cfg.device_budget;
        uint64_t busy = 0;
        for (auto& sp : s->slots)
            if (sp->busy) busy += slot_bytes(*sp);
        const uint64_t keep = slot->views.count(g) ? slot->view_bytes[g] : 0;
        const uint64_t vc = slot->views.count(g) ? 0 : workspace_estimate(g);
        // batch size: up to max_batch BFS queries of this graph, fewer if their
        // level rows (k * n * 4 bytes) would not fit beside everything running
        uint32_t kmax = 1;
        if (head->kind == EMOGI_QUERY_BFS) {
            kmax = s->cfg.max_batch ? s->cfg.max_batch : EMOGI_MAX_SOURCES;
            if (B) {
                const uint64_t base = busy + keep + vc;
                const uint64_t spare = B > base ? B - base : 0;
                kmax = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(kmax, spare / (4 * n)));
            }
        }
        auto job = std::make_unique<Job>();
        job->g = g;
        job->kind = head->kind;
        for (auto it = s->pending.begin(); it != s->pending.end() && job->reqs.size() < kmax;) {
            if ((*it)->g == g && (*it)->kind == head->kind) {
                job->reqs.push_back(*it);
                it = s->pending.erase(it);
            } else {
                ++it;
            }
        }
        const uint32_t k = (uint32_t)job->reqs.size();
        const bool rows_on_device = k > 1 || !head->out;
        const uint64_t rows = rows_on_device ? (uint64_t)k * n * 4 : 0;
        auto need = [&] { return vc + (rows > slot->dbuf_bytes ? rows - slot->dbuf_bytes : 0); };
        if (B && s->bytes_in_use + need() > B) {
            for (auto& sp : s->slots)  // other idle workers first
                if (sp.get() != slot && !sp->busy && s->bytes_in_use + need() > B) evict(s, *sp, nullptr);
            if (s->bytes_in_use + need() > B) evict(s, *slot, g);
        }
        if (B && s->bytes_in_use + need() > B) {
            if (s->in_flight == 0) {  // nothing will free memory: this job can never fit
                for (auto& r : job->reqs) {
                    finish_request(s, r, EMOGI_E_BUDGET, k, 0, 0, Clock::now());
                    r->done = true;
                }
                s->cv_done.notify_all();
                continue;
            }
            for (auto it = job->reqs.rbegin(); it != job->reqs.rend(); ++it) s->pending.push_front(*it);
            s->cv_sched.wait(lk);  // a finishing job wakes us
            continue;
        }
        // charge what the worker will create: its share's buffers and the grown row buffer
        s->bytes_in_use += need();
        if (vc) slot->view_bytes[g] = vc;
        job->bytes = 0;
        slot->busy = true;
        s->in_flight += k;
        slot->job = std::move(job);
        s->cv_sched.notify_all();
    }
}

}  // namespace

extern "C" {

emogi_status emogi_server_create(const emogi_server_config* cfg, emogi_server* out) {
    clear_error();
    if (!out) return fail(EMOGI_E_ARG, "out is NULL");
    *out = nullptr;
    emogi_server s = new (std::nothrow) emogi_server_s();
    if (!s) return fail(EMOGI_E_NOMEM, "server handle");
    if (cfg) {
        if (cfg->struct_size < sizeof(emogi_server_config)) {
            delete s;
            return fail(EMOGI_E_ARG, "emogi_server_config.struct_size too small");
        }
        s->cfg = *cfg;
    }
    if (!s->cfg.max_slots) s->cfg.max_slots = 4;
    if (s->cfg.max_slots > 64) s->cfg.max_slots = 64;
    if (s->cfg.max_batch > EMOGI_MAX_SOURCES) s->cfg.max_batch = EMOGI_MAX_SOURCES;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return fail(EMOGI_E_CUDA, "no CUDA device");
    }
    for (uint32_t i = 0; i < s->cfg.max_slots; i++) s->slots.push_back(std::make_unique<Slot>());
    for (auto& sp : s->slots) sp->th = std::thread(worker_main, s, sp.get());
    s->scheduler = std::thread(scheduler_main, s);
    *out = s;
    return EMOGI_OK;
}

emogi_status emogi_server_submit(emogi_server s, emogi_graph g, uint32_t kind, uint64_t src, uint32_t* out,
                                 uint64_t* ticket) {
    clear_error();
    if (!s || !g || !ticket) return fail(EMOGI_E_ARG, "server, graph and ticket must be non-NULL");
    if (kind != EMOGI_QUERY_BFS && kind != EMOGI_QUERY_SSSP) return fail(EMOGI_E_ARG, "unknown query kind %u", kind);
    if (src >= g->n) return fail(EMOGI_E_ARG, "source %llu is not below n = %llu", (unsigned long long)src,
                                 (unsigned long long)g->n);
    if (kind == EMOGI_QUERY_SSSP && !g->w) return fail(EMOGI_E_UNSUPPORTED, "SSSP query on a graph without weights");
    auto r = std::make_shared<Request>();
    r->g = g;
    r->kind = kind;
    r->src = src;
    r->out = out;
    r->submitted = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return fail(EMOGI_E_ARG, "server is shutting down");
    r->ticket = s->next_ticket++;
    s->by_ticket[r->ticket] = r;
    s->pending.push_back(r);
    *ticket = r->ticket;
    s->cv_sched.notify_all();
    return EMOGI_OK;
}

emogi_status emogi_server_wait(emogi_server s, uint64_t ticket, uint64_t timeout_ns, emogi_query_result* res) {
    clear_error();
    if (!s) return fail(EMOGI_E_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->by_ticket.find(ticket);
    if (it == s->by_ticket.end()) return fail(EMOGI_E_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    auto r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_ns == 0) {
        s->cv_done.wait(lk, ready);
    } else if (!s->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), ready)) {
        return fail(EMOGI_E_TIMEOUT, "query %llu not finished within %llu ns", (unsigned long long)ticket,
                    (unsigned long long)timeout_ns);
    }
    if (res) *res = r->res;
    s->by_ticket.erase(it);
    if (r->res.status != EMOGI_OK)
        return fail(r->res.status, "query %llu failed (%s)", (unsigned long long)ticket,
                    emogi_status_string(r->res.status));
    return EMOGI_OK;
}

emogi_status emogi_server_drain(emogi_server s) {
    if (!s) return fail(EMOGI_E_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->pending.empty() && s->in_flight == 0; });
    return EMOGI_OK;
}

uint64_t emogi_server_device_bytes(emogi_server s) {
    if (!s) return 0;
    std::lock_guard<std::mutex> lk(s->mu);
    return s->bytes_in_use;
}

emogi_status emogi_server_destroy(emogi_server s) {
    if (!s) return EMOGI_OK;
    emogi_server_drain(s);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
        s->cv_sched.notify_all();
    }
    if (s->scheduler.joinable()) s->scheduler.join();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->cv_sched.notify_all();
    }
    for (auto& sp : s->slots)
        if (sp->th.joinable()) sp->th.join();
    cudaSetDevice(s->device);
    for (auto& sp : s->slots) {
        for (auto& kv : sp->views) emogi_free_graph(kv.second);
        if (sp->dbuf) dev_free(sp->dbuf, sp->dbuf_bytes);
    }
    delete s;
    return EMOGI_OK;
}

}  // extern "C"
