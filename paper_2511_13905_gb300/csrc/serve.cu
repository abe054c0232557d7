// serve.cu -- the serving loop of include/pgdto.h: design sessions with device-resident
// state, HBM-budget admission, input upload on a copy stream, and continuous batching (a
// service thread launches everything that is ready while newer requests queue for the
// next cycle).  Inputs are copied by DMA straight from the caller's memory (the copy
// engine reads pageable memory at full speed on a coherent CPU-GPU link, so there is no
// host-side staging copy); each launch unit's reports and results are read as soon as
// that unit's event completes.  Host code only; the steps run in the kernels of
// seg_kernels.cu / coupled_kernels.cu through the public entry points.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pgdto.h"
#include "handle_internal.h"

namespace {

struct Session {
    uint64_t id = 0;
    int64_t n = 0;
    int m = 0;
    int64_t a_len = 0;
    bool coupled = false;
    pgdto_handle* h = nullptr;
    float* x = nullptr;       // device design (persists across steps)
    float* g = nullptr;       // device staging of grad f
    float* A = nullptr;       // device staging of the constraint gradients
    pgdto_info_slot* slot = nullptr;  // pinned: the last step's report
    cudaEvent_t uploaded = nullptr;
    uint64_t bytes = 0;
    bool busy = false;        // a step is queued or running
    bool closing = false;
};

struct Request {
    uint64_t ticket = 0;
    Session* s = nullptr;
    double g_val[4] = {0, 0, 0, 0};
    double G[4] = {0, 0, 0, 0};
    float* x_out = nullptr;
    bool close = false;
};

struct Done {
    pgdto_status status = PGDTO_OK;
    pgdto_info info;
    int64_t t_us = 0;  // completion on the server's clock
};

// One launch unit of a cycle (the batched group, or one session's own launch) and the
// event recorded behind it; the completion thread finishes units in launch order.
struct Unit {
    cudaEvent_t ev = nullptr;
    std::vector<Request> reqs;
};

}  // namespace

struct pgdto_server {
    uint64_t budget = 0, in_use = 0;
    int max_sessions = 0;
    pgdto_params params;
    cudaStream_t stream = nullptr;  // launches and result copies
    cudaStream_t copy = nullptr;    // input uploads
    cudaStream_t dtoh = nullptr;    // result downloads
    std::vector<cudaEvent_t> free_events;  // recorded behind launch units, recycled when finished
    std::vector<cudaEvent_t> all_events;
    std::mutex mu;
    std::condition_variable cv;       // service thread: work queued
    std::condition_variable cv_done;  // waiters: a result was published
    std::condition_variable cv_fin;   // completion thread: a unit was launched
    std::deque<Unit> inflight;        // launched, not yet finished (launch order)
    std::thread finisher;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    std::thread worker;
    bool stop = false;
    bool fin_stop = false;            // the service thread has stopped: finish what is in flight
    uint64_t next_ticket = 1;
    std::map<uint64_t, Session*> sessions;
    std::deque<Request> pending;
    std::vector<Request> running;     // every request launched and not yet published
    std::map<uint64_t, Done> done;
    int64_t batches = 0, steps = 0;
};

namespace {

int64_t clock_us(const pgdto_server* srv) {
    return std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - srv->t0).count();
}

uint64_t session_bytes(int64_t n, int64_t a_len) {
    // handle: x_prev, g_prev, d[2], z, z_lo (6 n floats) + workspace; session: x, g, A
    return (uint64_t)(6 * n + 2 * n + a_len) * sizeof(float) + (uint64_t)(3u << 20);
}

void free_session(Session* s) {
    if (!s) return;
    pgdto_destroy(s->h);
    cudaFree(s->x);
    cudaFree(s->g);
    cudaFree(s->A);
    cudaFreeHost(s->slot);
    if (s->uploaded) cudaEventDestroy(s->uploaded);
    delete s;
}

// Complete one launch unit: wait for its event, copy the designs to the callers' buffers,
// publish the reports (poll sees them at once), release closing sessions, recycle the event.
void finish_unit(pgdto_server* srv, Unit& unit) {
    cudaEventSynchronize(unit.ev);
    std::vector<Done> results(unit.reqs.size());
    cudaStreamWaitEvent(srv->dtoh, unit.ev, 0);
    for (size_t i = 0; i < unit.reqs.size(); ++i) {
        Request& r = unit.reqs[i];
        memset(&results[i].info, 0, sizeof(results[i].info));
        results[i].status = pgdto_info_collect(r.s->h, r.s->slot, &results[i].info);
        if (r.x_out &&
            cudaMemcpyAsync(r.x_out, r.s->x, (size_t)r.s->n * sizeof(float), cudaMemcpyDeviceToHost, srv->dtoh) !=
                cudaSuccess)
            results[i].status = PGDTO_ERR_CUDA;
    }
    if (cudaStreamSynchronize(srv->dtoh) != cudaSuccess)
        for (Done& d : results) d.status = PGDTO_ERR_CUDA;
    const int64_t now = clock_us(srv);
    for (Done& d : results) d.t_us = now;
    std::vector<Session*> closed;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        for (size_t i = 0; i < unit.reqs.size(); ++i) {
            Request& r = unit.reqs[i];
            srv->done[r.ticket] = results[i];
            r.s->busy = false;
            for (size_t q = 0; q < srv->running.size(); ++q)
                if (srv->running[q].ticket == r.ticket) {
                    srv->running.erase(srv->running.begin() + q);
                    break;
                }
            if (r.close) {
                srv->in_use -= r.s->bytes;
                srv->sessions.erase(r.s->id);
                closed.push_back(r.s);
            }
            srv->steps += 1;
        }
        srv->free_events.push_back(unit.ev);
    }
    srv->cv_done.notify_all();
    // device memory is released outside the lock (freeing waits for the device)
    for (Session* c : closed) free_session(c);
}

cudaEvent_t take_event(pgdto_server* srv) {
    std::lock_guard<std::mutex> lock(srv->mu);
    if (srv->free_events.empty()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        srv->all_events.push_back(e);
        return e;
    }
    cudaEvent_t e = srv->free_events.back();
    srv->free_events.pop_back();
    return e;
}

// One cycle: every small single/independent session in one batched step (pgdto_step_many:
// one thread-block cluster per session, sized by its n, all side by side), then each
// coupled session and each single/independent session whose handle runs on the whole GPU
// (n beyond the cluster range) in a launch of its own, smallest first.  A lone batched
// session runs through pgdto_step as well.  The launches are enqueued and handed to the
// completion thread, which reports each unit as soon as its own event completes, while
// this thread goes on to launch the next cycle.
void run_cycle(pgdto_server* srv, std::vector<Request>& batch) {
    std::vector<Request> group;
    std::vector<Request> own;
    for (Request& r : batch)
        (r.s->coupled || pgdto_handle_whole_gpu(r.s->h) ? own : group).push_back(r);
    if (group.size() == 1) {
        own.push_back(group[0]);
        group.clear();
    }
    std::sort(own.begin(), own.end(), [](const Request& a, const Request& b) { return a.s->n < b.s->n; });
    for (Request& r : batch) cudaStreamWaitEvent(srv->stream, r.s->uploaded, 0);
    std::vector<Unit> units;
    if (!group.empty()) {
        std::vector<pgdto_handle*> hs;
        std::vector<float*> xs;
        std::vector<const float*> gs, As;
        std::vector<double> gv, GG;
        for (Request& r : group) {
            hs.push_back(r.s->h);
            xs.push_back(r.s->x);
            gs.push_back(r.s->g);
            As.push_back(r.s->A);
            for (int j = 0; j < 4; ++j) {
                gv.push_back(r.g_val[j]);
                GG.push_back(r.G[j]);
            }
        }
        pgdto_step_many((int)hs.size(), hs.data(), xs.data(), gs.data(), As.data(), gv.data(), GG.data(), nullptr);
        for (Request& r : group) pgdto_info_enqueue(r.s->h, r.s->slot);
        Unit u;
        u.ev = take_event(srv);
        u.reqs = group;
        cudaEventRecord(u.ev, srv->stream);
        units.push_back(u);
    }
    for (Request& r : own) {
        pgdto_step(r.s->h, r.s->x, r.s->g, r.s->A, r.g_val, r.G, nullptr);
        pgdto_info_enqueue(r.s->h, r.s->slot);
        Unit u;
        u.ev = take_event(srv);
        u.reqs.assign(1, r);
        cudaEventRecord(u.ev, srv->stream);
        units.push_back(u);
    }
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->batches += (int64_t)units.size();
        for (Unit& u : units) srv->inflight.push_back(u);
    }
    srv->cv_fin.notify_one();
    batch.clear();
}

void service(pgdto_server* srv) {
    std::vector<Request> batch;
    for (;;) {
        {
            std::unique_lock<std::mutex> lock(srv->mu);
            srv->cv.wait(lock, [&] { return srv->stop || !srv->pending.empty(); });
            if (srv->pending.empty() && srv->stop) return;
            // everything queued now joins this cycle (one step per session: submit enforces it)
            while (!srv->pending.empty()) {
                batch.push_back(srv->pending.front());
                srv->running.push_back(srv->pending.front());
                srv->pending.pop_front();
            }
        }
        run_cycle(srv, batch);
    }
}

// The completion thread: finishes launched units in launch order (one stream, so that is
// also their completion order) until the server stops and nothing is in flight.
void finisher(pgdto_server* srv) {
    for (;;) {
        Unit u;
        {
            std::unique_lock<std::mutex> lock(srv->mu);
            srv->cv_fin.wait(lock, [&] { return srv->fin_stop || !srv->inflight.empty(); });
            if (srv->inflight.empty()) return;
            u = srv->inflight.front();
            srv->inflight.pop_front();
        }
        finish_unit(srv, u);
    }
}

// Admit and create a session (the caller holds the server's lock): the handle, the device
// design and input staging, the pinned report slot.  PGDTO_ERR_BUSY when the session limit
// or the HBM budget would be exceeded.
pgdto_status create_session(pgdto_server* srv, const pgdto_request* req, Session** out) {
    if (!req->x0) return PGDTO_ERR_ARG;
    const bool coupled = req->m > 1 && !req->seg_offsets;
    const int64_t a_len = coupled || (req->m == 1) ? req->n * (int64_t)req->m : req->n;
    const uint64_t bytes = session_bytes(req->n, a_len);
    if ((int)srv->sessions.size() >= srv->max_sessions || srv->in_use + bytes > srv->budget)
        return PGDTO_ERR_BUSY;
    Session* s = new Session();
    s->id = req->session;
    s->n = req->n;
    s->m = req->m;
    s->a_len = a_len;
    s->coupled = coupled;
    s->bytes = bytes;
    pgdto_params p = srv->params;
    p.mode = PGDTO_AUTO;
    p.eq_mask = req->eq_mask;
    if (coupled) p.engine = 0;  // coupled rows run on the grid engine (one launch each)
    pgdto_status st = pgdto_create(&s->h, req->n, req->m, req->seg_offsets, req->lo, req->hi, &p, srv->stream);
    const size_t nb = (size_t)req->n * sizeof(float);
    if (st == PGDTO_OK && (cudaMalloc(&s->x, nb) != cudaSuccess || cudaMalloc(&s->g, nb) != cudaSuccess ||
                           cudaMalloc(&s->A, (size_t)a_len * sizeof(float)) != cudaSuccess ||
                           cudaMallocHost(&s->slot, sizeof(pgdto_info_slot)) != cudaSuccess ||
                           cudaEventCreateWithFlags(&s->uploaded, cudaEventDisableTiming) != cudaSuccess))
        st = PGDTO_ERR_OOM;
    if (st == PGDTO_OK) st = pgdto_set_state(s->h, nullptr, nullptr, nullptr, 0);
    if (st != PGDTO_OK) {
        free_session(s);
        return st == PGDTO_ERR_OOM ? PGDTO_ERR_BUSY : st;
    }
    srv->sessions[s->id] = s;
    srv->in_use += bytes;
    *out = s;
    return PGDTO_OK;
}

}  // namespace

extern "C" pgdto_status pgdto_server_create(pgdto_server** out, uint64_t budget_bytes, int max_sessions,
                                            const pgdto_params* params, void* cuda_stream) {
    if (!out || max_sessions < 1) return PGDTO_ERR_ARG;
    *out = nullptr;
    pgdto_server* srv = new pgdto_server();
    srv->budget = budget_bytes;
    srv->max_sessions = max_sessions;
    if (params) srv->params = *params;
    else pgdto_params_default(&srv->params);
    srv->stream = (cudaStream_t)cuda_stream;
    if (cudaStreamCreateWithFlags(&srv->copy, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&srv->dtoh, cudaStreamNonBlocking) != cudaSuccess) {
        if (srv->copy) cudaStreamDestroy(srv->copy);
        if (srv->dtoh) cudaStreamDestroy(srv->dtoh);
        delete srv;
        return PGDTO_ERR_CUDA;
    }
    srv->worker = std::thread(service, srv);
    srv->finisher = std::thread(finisher, srv);
    *out = srv;
    return PGDTO_OK;
}

extern "C" pgdto_status pgdto_submit(pgdto_server* srv, const pgdto_request* req, uint64_t* ticket) {
    if (!srv || !req || !ticket || !req->grad_f || !req->A || req->n < 1 || req->m < 1 || req->m > 4)
        return PGDTO_ERR_ARG;
    std::unique_lock<std::mutex> lock(srv->mu);
    Session* s = nullptr;
    bool fresh = false;
    auto it = srv->sessions.find(req->session);
    if (it != srv->sessions.end()) {
        s = it->second;
        if (s->n != req->n || s->m != req->m) return PGDTO_ERR_ARG;
        if (s->busy) return PGDTO_ERR_BUSY;
    } else {
        pgdto_status cst = create_session(srv, req, &s);
        if (cst != PGDTO_OK) return cst;
        fresh = true;
    }
    // the session is reserved (busy) while its inputs upload outside the lock, so other
    // submits, polls and the service thread carry on meanwhile
    s->busy = true;
    lock.unlock();
    // DMA from the caller's buffers on the copy stream, waited for before returning, so the
    // buffers are free on return whether they are pageable or pinned
    const size_t nb = (size_t)s->n * sizeof(float);
    cudaError_t e = cudaSuccess;
    if (fresh) e = cudaMemcpyAsync(s->x, req->x0, nb, cudaMemcpyHostToDevice, srv->copy);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->g, req->grad_f, nb, cudaMemcpyHostToDevice, srv->copy);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->A, req->A, (size_t)s->a_len * sizeof(float), cudaMemcpyHostToDevice, srv->copy);
    if (e == cudaSuccess) e = cudaEventRecord(s->uploaded, srv->copy);
    if (e == cudaSuccess) e = cudaEventSynchronize(s->uploaded);
    lock.lock();
    if (e != cudaSuccess) {
        s->busy = false;
        if (fresh) {
            srv->in_use -= s->bytes;
            srv->sessions.erase(s->id);
            free_session(s);
        }
        return PGDTO_ERR_CUDA;
    }
    Request r;
    r.ticket = srv->next_ticket++;
    r.s = s;
    for (int j = 0; j < req->m; ++j) {
        r.g_val[j] = req->g_val[j];
        r.G[j] = req->G[j];
    }
    r.x_out = req->x_out;
    r.close = req->close_session != 0;
    srv->pending.push_back(r);
    *ticket = r.ticket;
    lock.unlock();
    srv->cv.notify_one();
    return PGDTO_OK;
}

extern "C" pgdto_status pgdto_server_open(pgdto_server* srv, const pgdto_request* req) {
    if (!srv || !req || !req->x0 || req->n < 1 || req->m < 1 || req->m > 4) return PGDTO_ERR_ARG;
    std::unique_lock<std::mutex> lock(srv->mu);
    if (srv->sessions.count(req->session)) return PGDTO_ERR_ARG;
    Session* s = nullptr;
    pgdto_status st = create_session(srv, req, &s);
    if (st != PGDTO_OK) return st;
    s->busy = true;  // reserved while the design uploads outside the lock
    lock.unlock();
    cudaError_t e = cudaMemcpyAsync(s->x, req->x0, (size_t)s->n * sizeof(float), cudaMemcpyHostToDevice, srv->copy);
    if (e == cudaSuccess) e = cudaEventRecord(s->uploaded, srv->copy);
    if (e == cudaSuccess) e = cudaEventSynchronize(s->uploaded);
    lock.lock();
    s->busy = false;
    if (e != cudaSuccess) {
        srv->in_use -= s->bytes;
        srv->sessions.erase(s->id);
        lock.unlock();
        free_session(s);
        return PGDTO_ERR_CUDA;
    }
    return PGDTO_OK;
}

extern "C" pgdto_status pgdto_poll(pgdto_server* srv, uint64_t ticket, pgdto_status* done, pgdto_info* info) {
    if (!srv || !done) return PGDTO_ERR_ARG;
    std::lock_guard<std::mutex> lock(srv->mu);
    auto it = srv->done.find(ticket);
    if (it != srv->done.end()) {
        *done = it->second.status;
        if (info) *info = it->second.info;
        srv->done.erase(it);
        return PGDTO_OK;
    }
    for (const Request& r : srv->pending)
        if (r.ticket == ticket) {
            *done = PGDTO_ERR_BUSY;
            return PGDTO_OK;
        }
    for (const Request& r : srv->running)
        if (r.ticket == ticket) {
            *done = PGDTO_ERR_BUSY;
            return PGDTO_OK;
        }
    return PGDTO_ERR_ARG;  // unknown or already reported
}

extern "C" pgdto_status pgdto_wait(pgdto_server* srv, uint64_t ticket, int timeout_ms, pgdto_status* done,
                                   pgdto_info* info, int64_t* completed_us) {
    if (!srv || !done || timeout_ms < 0) return PGDTO_ERR_ARG;
    std::unique_lock<std::mutex> lock(srv->mu);
    auto known = [&] {
        for (const Request& r : srv->pending)
            if (r.ticket == ticket) return true;
        for (const Request& r : srv->running)
            if (r.ticket == ticket) return true;
        return false;
    };
    const auto until = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        auto it = srv->done.find(ticket);
        if (it != srv->done.end()) {
            *done = it->second.status;
            if (info) *info = it->second.info;
            if (completed_us) *completed_us = it->second.t_us;
            srv->done.erase(it);
            return PGDTO_OK;
        }
        if (!known()) return PGDTO_ERR_ARG;  // unknown or already reported
        if (srv->cv_done.wait_until(lock, until) == std::cv_status::timeout && srv->done.count(ticket) == 0) {
            *done = PGDTO_ERR_BUSY;
            return PGDTO_OK;
        }
    }
}

extern "C" int64_t pgdto_server_clock_us(const pgdto_server* srv) { return srv ? clock_us(srv) : -1; }

extern "C" pgdto_status pgdto_server_stats(pgdto_server* srv, int64_t* batches, int64_t* steps, int* sessions,
                                           uint64_t* bytes_in_use) {
    if (!srv) return PGDTO_ERR_ARG;
    std::lock_guard<std::mutex> lock(srv->mu);
    if (batches) *batches = srv->batches;
    if (steps) *steps = srv->steps;
    if (sessions) *sessions = (int)srv->sessions.size();
    if (bytes_in_use) *bytes_in_use = srv->in_use;
    return PGDTO_OK;
}

extern "C" void pgdto_server_destroy(pgdto_server* srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->stop = true;
    }
    srv->cv.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->fin_stop = true;
    }
    srv->cv_fin.notify_all();
    if (srv->finisher.joinable()) srv->finisher.join();
    cudaStreamSynchronize(srv->stream);
    for (auto& kv : srv->sessions) free_session(kv.second);
    srv->sessions.clear();
    for (cudaEvent_t e : srv->all_events) cudaEventDestroy(e);
    cudaStreamDestroy(srv->copy);
    cudaStreamDestroy(srv->dtoh);
    delete srv;
}
