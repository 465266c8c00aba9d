// Serving form: a request loop that renders novel views of mixed resolution and view count as
// they arrive, from input pyramids kept resident per time step.
//
// Threads.  quark_serve_submit / poll / cancel / stats may be called from any host thread; one
// scheduler thread owns the context's launches.  Requests wait in a FIFO queue; the scheduler
// admits the head of the queue as soon as a slot (a CUDA stream of its own) is free and the
// request's device footprint fits under the HBM cap next to the resident pyramids, so requests
// that arrive while others run start as slots and memory free up and their kernels overlap on
// the device.  Each request's LDM comes from the stream-ordered allocator on its slot's stream
// and returns to it when the request's work is done, so admission never stalls other streams.
// Completion is detected by polling one event per slot.  A request's result does not depend on
// what else runs: the same kernels run on the same inputs with the same launch shapes.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "api_internal.h"

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum TicketState { T_PENDING, T_RUNNING, T_DONE, T_CANCELLED };

struct Ticket {
    quark_request req{};
    TicketState state = T_PENDING;
    quark_status status = QUARK_OK;
    double t_submit = 0, t_admit = 0, t_done = 0;
    size_t bytes = 0;
    int host_out = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    uint64_t ticket = 0;
    quark_ldm* ldm = nullptr;
};

bool device_pointer(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

struct quark_server {
    quark_ctx* ctx = nullptr;
    quark_serve_config cfg{};
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Ticket> tickets;
    std::vector<Slot> slots;
    std::map<int, quark_pyramid*> steps;
    size_t steps_bytes = 0;
    size_t in_use = 0, high_water = 0;
    uint64_t next_ticket = 1;
    uint64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, rejected = 0;
    std::vector<double> latencies_ms;
    double t_start = 0, t_first_done = 0, t_last_done = 0;
    bool stop = false, paused = false;
    cudaStream_t setup = nullptr;
    std::thread th;
};

static size_t pyramid_bytes(const quark_pyramid* p) {
    size_t b = p->rgba_bytes + p->staging_bytes;
    for (int i = 0; i < 4; ++i) b += p->level_bytes[i];
    return b;
}

// Runs on the scheduler thread with the lock held.
static void finish(quark_server* S, Slot& slot, quark_status st) {
    Ticket& t = S->tickets[slot.ticket];
    t.state = T_DONE;
    t.status = st;
    t.t_done = now_s();
    if (slot.ldm) {
        qk_ldm_free(slot.ldm);  // stream-ordered frees after the request's own work
        slot.ldm = nullptr;
    }
    S->in_use -= t.bytes;
    slot.busy = false;
    if (st == QUARK_OK) {
        S->completed++;
        S->latencies_ms.push_back((t.t_done - t.t_submit) * 1e3);
        if (S->completed == 1) S->t_first_done = t.t_done;
        S->t_last_done = t.t_done;
    } else {
        S->failed++;
    }
    S->cv_done.notify_all();
}

static quark_status launch_request(quark_server* S, Slot& slot, Ticket& t) {
    quark_ctx* ctx = S->ctx;
    auto it = S->steps.find(t.req.timestep);
    if (it == S->steps.end()) return qk_fail(ctx, QUARK_ENOTFOUND, "time step %d is not resident", t.req.timestep);
    quark_pyramid* pyr = it->second;
    quark_status s = qk_ldm_create(ctx, &t.req.target, t.req.n_views, slot.stream, &slot.ldm);
    for (int j = 0; s == QUARK_OK && j < ctx->cfg.n_scales; ++j)
        s = qk_update_fuse(ctx, pyr, t.req.n_views, j, slot.ldm, slot.stream);
    if (s == QUARK_OK) s = qk_render(ctx, slot.ldm, pyr, t.req.n_views, t.req.rgba, t.host_out, slot.stream);
    if (s == QUARK_OK) {
        cudaError_t e = cudaEventRecord(slot.done, slot.stream);
        if (e != cudaSuccess) s = qk_fail(ctx, QUARK_ECUDA, "cudaEventRecord: %s", cudaGetErrorString(e));
    }
    return s;
}

static void scheduler(quark_server* S) {
    cudaSetDevice(S->ctx->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        bool progress = false;
        bool running = false;
        for (Slot& slot : S->slots) {
            if (!slot.busy) continue;
            cudaError_t q = cudaEventQuery(slot.done);
            if (q == cudaErrorNotReady) {
                running = true;
                continue;
            }
            finish(S, slot, q == cudaSuccess ? QUARK_OK : QUARK_ECUDA);
            progress = true;
        }
        if (S->stop && S->pending.empty() && !running) break;
        while (!S->paused && !S->pending.empty()) {
            Ticket& t = S->tickets[S->pending.front()];
            Slot* free_slot = nullptr;
            for (Slot& slot : S->slots)
                if (!slot.busy) {
                    free_slot = &slot;
                    break;
                }
            if (!free_slot) break;
            const size_t cap = S->cfg.hbm_cap_bytes;
            if (cap && S->steps_bytes + S->in_use + t.bytes > cap) break;  // FIFO: the head waits for memory
            const uint64_t id = S->pending.front();
            S->pending.pop_front();
            t.state = T_RUNNING;
            t.t_admit = now_s();
            free_slot->busy = true;
            free_slot->ticket = id;
            S->in_use += t.bytes;
            S->high_water = std::max(S->high_water, S->steps_bytes + S->in_use);
            quark_status st = launch_request(S, *free_slot, t);
            if (st != QUARK_OK) {
                cudaStreamSynchronize(free_slot->stream);
                finish(S, *free_slot, st);
            }
            progress = true;
        }
        if (!progress) S->cv_sched.wait_for(lk, std::chrono::microseconds(50));
    }
}

extern "C" quark_status quark_serve_start(quark_ctx* ctx, const quark_serve_config* cfg, quark_server** out) {
    if (!ctx || !cfg || !out) return qk_fail(ctx, QUARK_EINVAL, "NULL argument");
    *out = nullptr;
    if (!ctx->weights_loaded) return qk_fail(ctx, QUARK_EINVAL, "weights not loaded");
    if (cfg->n_slots < 1 || cfg->n_slots > 64) return qk_fail(ctx, QUARK_EINVAL, "n_slots must be 1..64");
    if (cfg->queue_capacity < 1) return qk_fail(ctx, QUARK_EINVAL, "queue_capacity must be >= 1");
    cudaSetDevice(ctx->device);
    quark_server* S = new quark_server();
    S->ctx = ctx;
    S->cfg = *cfg;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;  // keep freed LDM memory in the pool between requests
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    S->slots.resize(cfg->n_slots);
    for (Slot& s : S->slots) {
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            for (Slot& t : S->slots) {
                if (t.stream) cudaStreamDestroy(t.stream);
                if (t.done) cudaEventDestroy(t.done);
            }
            delete S;
            return qk_fail(ctx, QUARK_ECUDA, "cannot create the slot streams");
        }
    }
    cudaStreamCreateWithFlags(&S->setup, cudaStreamNonBlocking);
    S->t_start = now_s();
    S->th = std::thread(scheduler, S);
    *out = S;
    return QUARK_OK;
}

extern "C" quark_status quark_serve_set_timestep(quark_server* S, int timestep, const float* images,
                                                 const quark_camera* cams, int V) {
    if (!S || !images || !cams) return qk_fail(S ? S->ctx : nullptr, QUARK_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> g(S->mu);
    for (auto& kv : S->tickets)
        if ((kv.second.state == T_PENDING || kv.second.state == T_RUNNING) && kv.second.req.timestep == timestep)
            return qk_fail(S->ctx, QUARK_EBUSY, "time step %d has requests queued or running", timestep);
    quark_pyramid* p = nullptr;
    auto it = S->steps.find(timestep);
    if (it != S->steps.end()) {
        p = it->second;
        if (p->V != V || p->H != cams[0].height || p->W != cams[0].width) {
            S->steps_bytes -= pyramid_bytes(p);
            quark_release_pyramid(p);
            S->steps.erase(it);
            p = nullptr;
        }
    }
    const bool fresh = p == nullptr;
    quark_status s = quark_encode_pyramid(S->ctx, images, cams, V, S->setup, &p);
    if (s != QUARK_OK) return s;
    cudaError_t e = cudaStreamSynchronize(S->setup);
    if (e != cudaSuccess) return qk_fail(S->ctx, QUARK_ECUDA, "encode: %s", cudaGetErrorString(e));
    if (fresh) {
        S->steps[timestep] = p;
        S->steps_bytes += pyramid_bytes(p);
        S->high_water = std::max(S->high_water, S->steps_bytes + S->in_use);
    }
    return QUARK_OK;
}

extern "C" quark_status quark_serve_submit(quark_server* S, const quark_request* req, uint64_t* ticket) {
    if (!S || !req || !ticket) return qk_fail(S ? S->ctx : nullptr, QUARK_EINVAL, "NULL argument");
    quark_ctx* ctx = S->ctx;
    const quark_config& c = ctx->cfg;
    quark_status s = qk_validate_camera(nullptr, req->target, "target");
    if (s != QUARK_OK) return s;
    for (int j = 0; j < c.n_scales; ++j)
        if (req->target.height % c.k[j] || req->target.width % c.k[j])
            return qk_fail(nullptr, QUARK_EINVAL, "output %dx%d not divisible by k=%d", req->target.width,
                           req->target.height, c.k[j]);
    if (!req->rgba) return qk_fail(nullptr, QUARK_EINVAL, "NULL output");
    const int host_out = device_pointer(req->rgba) ? 0 : 1;
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stop) return qk_fail(nullptr, QUARK_EINVAL, "server is stopping");
    auto it = S->steps.find(req->timestep);
    if (it == S->steps.end()) return qk_fail(nullptr, QUARK_ENOTFOUND, "time step %d is not resident", req->timestep);
    if (req->n_views < 1 || req->n_views > it->second->V)
        return qk_fail(nullptr, QUARK_EINVAL, "n_views %d outside 1..%d", req->n_views, it->second->V);
    Ticket t;
    t.req = *req;
    t.host_out = host_out;
    t.bytes = qk_ldm_bytes(c, req->target.width, req->target.height, req->n_views, host_out) + (1u << 20);
    if (S->cfg.hbm_cap_bytes && S->steps_bytes + t.bytes > S->cfg.hbm_cap_bytes) {
        S->rejected++;
        return qk_fail(nullptr, QUARK_ENOMEM, "request needs %zu bytes; the HBM cap leaves %zu beside the pyramids",
                       t.bytes, S->cfg.hbm_cap_bytes - std::min(S->cfg.hbm_cap_bytes, S->steps_bytes));
    }
    if ((int)S->pending.size() >= S->cfg.queue_capacity) {
        S->rejected++;
        return qk_fail(nullptr, QUARK_EBUSY, "queue full (%d pending)", (int)S->pending.size());
    }
    t.t_submit = now_s();
    const uint64_t id = S->next_ticket++;
    S->tickets[id] = t;
    S->pending.push_back(id);
    S->submitted++;
    *ticket = id;
    S->cv_sched.notify_one();
    return QUARK_OK;
}

extern "C" quark_status quark_serve_poll(quark_server* S, uint64_t ticket, int timeout_us, quark_result* out) {
    if (!S || !out) return qk_fail(S ? S->ctx : nullptr, QUARK_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return qk_fail(nullptr, QUARK_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    auto ready = [&] {
        auto i = S->tickets.find(ticket);
        return i != S->tickets.end() && (i->second.state == T_DONE || i->second.state == T_CANCELLED);
    };
    if (!ready()) {
        if (timeout_us <= 0) return QUARK_EAGAIN;
        if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready))
            return qk_fail(nullptr, QUARK_ETIMEDOUT, "ticket %llu not done within %d us", (unsigned long long)ticket,
                           timeout_us);
    }
    Ticket& t = S->tickets[ticket];
    out->status = t.state == T_CANCELLED ? QUARK_EINVAL : t.status;
    out->user_tag = t.req.user_tag;
    out->queue_ms = t.state == T_DONE ? (t.t_admit - t.t_submit) * 1e3 : 0.0;
    out->gpu_ms = t.state == T_DONE ? (t.t_done - t.t_admit) * 1e3 : 0.0;
    out->total_ms = t.state == T_DONE ? (t.t_done - t.t_submit) * 1e3 : 0.0;
    out->cancelled = t.state == T_CANCELLED;
    S->tickets.erase(ticket);
    return QUARK_OK;
}

extern "C" quark_status quark_serve_cancel(quark_server* S, uint64_t ticket) {
    if (!S) return qk_fail(nullptr, QUARK_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return qk_fail(nullptr, QUARK_ENOTFOUND, "unknown ticket");
    if (it->second.state != T_PENDING) return qk_fail(nullptr, QUARK_EBUSY, "ticket already admitted");
    S->pending.erase(std::find(S->pending.begin(), S->pending.end(), ticket));
    it->second.state = T_CANCELLED;
    S->cancelled++;
    S->cv_done.notify_all();
    return QUARK_OK;
}

extern "C" quark_status quark_serve_pause(quark_server* S, int paused) {
    if (!S) return qk_fail(nullptr, QUARK_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> g(S->mu);
    S->paused = paused != 0;
    S->cv_sched.notify_one();
    return QUARK_OK;
}

extern "C" quark_status quark_serve_stats(quark_server* S, quark_stats* out) {
    if (!S || !out) return qk_fail(nullptr, QUARK_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> g(S->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->failed = S->failed;
    out->cancelled = S->cancelled;
    out->rejected = S->rejected;
    out->queued = (int)S->pending.size();
    for (const Slot& s : S->slots) out->in_flight += s.busy ? 1 : 0;
    if (!S->latencies_ms.empty()) {
        std::vector<double> l = S->latencies_ms;
        std::sort(l.begin(), l.end());
        auto pct = [&](double p) { return l[std::min(l.size() - 1, (size_t)(p * (l.size() - 1) + 0.5))]; };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double sum = 0;
        for (double v : l) sum += v;
        out->mean_ms = sum / l.size();
    }
    const double span = S->t_last_done - S->t_start;
    out->fps = span > 0 ? S->completed / span : 0.0;
    out->hbm_in_use = S->steps_bytes + S->in_use;
    out->hbm_high_water = S->high_water;
    return QUARK_OK;
}

extern "C" quark_status quark_serve_stop(quark_server* S) {
    if (!S) return QUARK_OK;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        S->paused = false;
        for (uint64_t id : S->pending) {
            S->tickets[id].state = T_CANCELLED;
            S->cancelled++;
        }
        S->pending.clear();
        S->cv_sched.notify_one();
        S->cv_done.notify_all();
    }
    if (S->th.joinable()) S->th.join();
    cudaSetDevice(S->ctx->device);
    for (Slot& s : S->slots) {
        cudaStreamSynchronize(s.stream);
        cudaStreamDestroy(s.stream);
        cudaEventDestroy(s.done);
    }
    for (auto& kv : S->steps) quark_release_pyramid(kv.second);
    if (S->setup) cudaStreamDestroy(S->setup);
    delete S;
    return QUARK_OK;
}
