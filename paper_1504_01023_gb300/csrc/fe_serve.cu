// Serving loop: integration requests on resident meshes arrive at any time; a
// scheduler thread admits them under the HBM budget, merges waiting
// mixed-precision requests into batched launches (continuous batching), keeps
// up to serve_slots launches in flight on their own streams, and stamps each
// request's completion from a host callback on its stream.
//
// Launch policy: while less than kFeedElems elements are in flight, waiting
// requests launch at once (an idle or lightly loaded GPU adds no queueing delay);
// beyond that they accumulate until the work in flight drops below it, so that a
// loaded GPU runs fewer, larger launches. One launch takes at most kLaunchElems
// elements (the first request always fits), so completions keep arriving while
// later launches run.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <memory>

#include "fe_runtime.h"

namespace fe {

static double now_us() {
    using namespace std::chrono;
    return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
    fe_request r{};
    MeshRec mesh{};
    void *A = nullptr, *b = nullptr;
    uint8_t *flags = nullptr;
    uint64_t out_bytes = 0;
    double t_submit = 0, t_launch = 0, t_done = 0;
    fe_status status = FE_OK;
    int state = 0;  // 0 waiting, 1 running, 2 done
    int slot = -1;
    bool returned = false;  // handed out by fe_serve_wait_any
};

struct ServeState;

constexpr uint64_t kFeedElems = uint64_t(32) << 20;    // ~2 ms of GPU work (measured: 32M > 16M, 64M)
constexpr uint64_t kLaunchElems = uint64_t(16) << 20;   // measured: 16M > 32M, 64M for large requests
struct Slot {
    ServeState *owner = nullptr;
    cudaStream_t stream = nullptr;
    bool busy = false;                 // guarded by the state's mutex
    std::atomic<int> done{0};          // set by the stream's host callback
    double t_done = 0;                 // written by the callback before `done`
    std::vector<uint64_t> tickets;
    uint64_t elems = 0;                // elements of the launch in flight (mutex)
    bool launching = false;            // between admission and publication (mutex)
    DynBatch dyn;
    Scratch plain;
};

struct ServeState {
    fe_ctx *ctx = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    std::thread th;
    bool stop = false;
    std::deque<uint64_t> waiting;
    std::unordered_map<uint64_t, Req> reqs;
    // completion queue: finished tickets in completion order, each returned once
    // by fe_serve_wait_any; entries of released requests are skipped and, when
    // they pile up, compacted away (the queue stays O(live requests))
    std::deque<uint64_t> done_q;
    std::condition_variable done_cv;
    uint64_t next_ticket = 1;
    std::vector<std::unique_ptr<Slot>> slots;
    cudaMemPool_t pool = nullptr;
    uint64_t out_used = 0;
};

// Host callback at the end of a slot's work. It takes no lock (the scheduler may
// hold the mutex across CUDA calls that wait for the device): it stamps the time,
// publishes the flag and wakes the scheduler.
static void CUDART_CB on_slot_done(void *p) {
    Slot *sl = static_cast<Slot *>(p);
    sl->t_done = now_us();
    sl->done.store(1, std::memory_order_release);
    sl->owner->cv.notify_all();
}

// Mark the requests of finished slots done, in completion order, queue them for
// fe_serve_wait_any, and free the slots (lock held).
static void reap(ServeState *s) {
    Slot *fin[64];
    int nf = 0;
    for (auto &up : s->slots) {
        Slot &sl = *up;
        if (!sl.busy || sl.launching || !sl.done.load(std::memory_order_acquire)) continue;
        if (nf < 64) fin[nf++] = &sl;
    }
    std::sort(fin, fin + nf, [](const Slot *a, const Slot *b) { return a->t_done < b->t_done; });
    bool any = false;
    for (int f = 0; f < nf; ++f) {
        Slot &sl = *fin[f];
        for (uint64_t tk : sl.tickets) {
            auto it = s->reqs.find(tk);
            if (it != s->reqs.end()) {
                it->second.t_done = sl.t_done;
                it->second.state = 2;
                s->done_q.push_back(tk);
                any = true;
            }
        }
        sl.tickets.clear();
        sl.elems = 0;
        sl.done.store(0, std::memory_order_relaxed);
        sl.busy = false;
    }
    if (any) s->done_cv.notify_all();
    if (s->done_q.size() > 2 * s->reqs.size() + 4096) {
        std::deque<uint64_t> keep;
        for (uint64_t tk : s->done_q) {
            auto it = s->reqs.find(tk);
            if (it != s->reqs.end() && !it->second.returned) keep.push_back(tk);
        }
        s->done_q.swap(keep);
    }
}

static void fill_result(const Req &q, fe_result *res) {
    res->status = q.status;
    res->type = q.mesh.type;
    res->n_elem = q.mesh.n_elem;
    res->A = q.A;
    res->b = q.b;
    res->flags = q.flags;
    res->t_submit_us = q.t_submit;
    res->t_launch_us = q.t_launch;
    res->t_done_us = q.t_done;
}

static uint64_t out_bytes_of(const MeshRec &m, fe_precision prec) {
    const uint64_t ns = uint64_t(ns_of(m.type)), cs = prec == FE_FP32_MIXED ? 4 : 8;
    auto r256 = [](uint64_t v) { return (v + 255) / 256 * 256; };
    return r256(uint64_t(m.n_elem) * ns * ns * cs) + r256(uint64_t(m.n_elem) * ns * cs) + r256(uint64_t(m.n_elem));
}

// One admitted request as the launching code sees it, outside the lock.
struct Job {
    uint64_t ticket;
    fe_request r;
    MeshRec mesh;
    void *A = nullptr, *b = nullptr;
    uint8_t *flags = nullptr;
    fe_status status = FE_OK;
};

// Allocate the outputs of the jobs and launch them on the slot's stream: mixed
// requests as one batched launch, the others as their own launches; then the
// slot's completion callback. Runs without the lock (it makes CUDA calls, which
// may wait); touches only the jobs and the slot's own stream and tables.
static void launch_jobs(ServeState *s, Slot &sl, std::vector<Job> &jobs) {
    TraceRange tr("serve launch");
    fe_ctx *ctx = s->ctx;
    std::vector<BatchItemDev> items;
    for (Job &j : jobs) {
        const MeshRec &m = j.mesh;
        // outputs from the context's stream-ordered pool: one allocation holding
        // A, b and the flags, each part on a 256-byte boundary
        const uint64_t ns = ns_of(m.type), cs = j.r.prec == FE_FP32_MIXED ? 4 : 8;
        auto r256 = [](uint64_t v) { return (v + 255) / 256 * 256; };
        const uint64_t bA = r256(uint64_t(m.n_elem) * ns * ns * cs), bB = r256(uint64_t(m.n_elem) * ns * cs);
        void *base = nullptr;
        cudaError_t e = take_alloc_fault(ctx)   // an injected fault fails it as out of memory
                            ? cudaErrorMemoryAllocation
                            : cudaMallocFromPoolAsync(&base, bA + bB + r256(uint64_t(m.n_elem)), s->pool, sl.stream);
        if (e != cudaSuccess) {
            j.status = cuda_check(ctx, e, "cudaMallocFromPoolAsync(serve outputs)");
            continue;
        }
        j.A = base;
        j.b = static_cast<unsigned char *>(base) + bA;
        j.flags = static_cast<uint8_t *>(base) + bA + bB;
        if (j.r.prec == FE_FP32_MIXED) {
            BatchItemDev d;
            memset(&d, 0, sizeof d);
            d.p.n = m.n_elem;
            d.p.X = m.coords;
            d.p.xs = m.n_elem;
            d.p.C = j.r.coefs;
            d.p.cs = m.n_elem;
            d.p.A = j.A;
            d.p.B = j.b;
            d.p.os = m.n_elem;
            d.p.flags = j.flags;
            d.p.item = unsigned(items.size());
            d.combo = batch_combo(m.type, j.r.kind, j.r.quad, j.r.coef_mode == FE_COEF_PER_QPOINT);
            items.push_back(d);
        } else {
            fe_elem_args a{};
            a.n_elem = m.n_elem;
            a.coords = m.coords;
            a.coords_layout = FE_LAYOUT_AOS;
            a.kind = j.r.kind;
            a.quad = j.r.quad;
            a.coef_mode = j.r.coef_mode;
            a.coefs = j.r.coefs;
            a.coefs_layout = FE_LAYOUT_AOS;
            a.prec = j.r.prec;
            a.memory = FE_MEM_DEVICE;
            fe_out o{};
            o.A = j.A;
            o.b = j.b;
            o.layout = FE_LAYOUT_AOS;
            o.flags = j.flags;
            o.memory = FE_MEM_DEVICE;
            const Shape sh = default_shape(m.type);
            j.status = launch_set(ctx, m.type, &a, &o, sl.plain, sl.stream, &sh);
        }
    }
    if (!items.empty()) {
        const fe_status st = dyn_batch_launch(ctx, sl.dyn, items, sl.stream);
        if (st != FE_OK)
            for (Job &j : jobs)
                if (j.r.prec == FE_FP32_MIXED && j.status == FE_OK) j.status = st;
    }
    cudaLaunchHostFunc(sl.stream, on_slot_done, &sl);
}

// Launch an admitted batch into a free slot. Called with the lock held; releases
// it around the CUDA calls. While the slot is `launching`, reap leaves it alone
// (its callback may fire before the results are published); a running request
// cannot be released, so its record stays in place meanwhile.
static void launch_slot(ServeState *s, int si, std::vector<uint64_t> &batch, std::unique_lock<std::mutex> &lk) {
    Slot &sl = *s->slots[si];
    sl.busy = true;
    sl.launching = true;
    sl.elems = 0;
    std::vector<Job> jobs;
    jobs.reserve(batch.size());
    const double t = now_us();
    for (uint64_t tk : batch) {
        Req &q = s->reqs[tk];
        q.t_launch = t;
        q.state = 1;
        q.slot = si;
        sl.elems += uint64_t(q.mesh.n_elem);
        Job j;
        j.ticket = tk;
        j.r = q.r;
        j.mesh = q.mesh;
        jobs.push_back(j);
    }
    lk.unlock();
    launch_jobs(s, sl, jobs);
    lk.lock();
    for (const Job &j : jobs) {
        Req &q = s->reqs[j.ticket];
        q.A = j.A;
        q.b = j.b;
        q.flags = j.flags;
        q.status = j.status;
    }
    sl.tickets = batch;
    sl.launching = false;
}

static void scheduler(ServeState *s) {
    cudaSetDevice(s->ctx->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        reap(s);
        // admit waiting requests in arrival order while the budget allows
        int free_slot = -1;
        uint64_t in_flight = 0;
        for (size_t i = 0; i < s->slots.size(); ++i) {
            if (!s->slots[i]->busy) {
                if (free_slot < 0) free_slot = int(i);
            } else {
                in_flight += s->slots[i]->elems;
            }
        }
        if (free_slot >= 0 && !s->waiting.empty() && in_flight < kFeedElems) {
            std::vector<uint64_t> batch;
            uint64_t elems = 0;
            const uint64_t resident = s->ctx->hbm_used.load();
            while (!s->waiting.empty()) {
                Req &q = s->reqs[s->waiting.front()];
                if (resident + s->out_used + q.out_bytes > s->ctx->hbm_budget) break;  // wait for releases
                if (!batch.empty() && elems + uint64_t(q.mesh.n_elem) > kLaunchElems) break;
                s->out_used += q.out_bytes;
                elems += uint64_t(q.mesh.n_elem);
                batch.push_back(s->waiting.front());
                s->waiting.pop_front();
            }
            if (!batch.empty()) {
                launch_slot(s, free_slot, batch, lk);
                continue;
            }
        }
        s->cv.wait_for(lk, std::chrono::milliseconds(2));
    }
}

void serve_destroy(fe_ctx *ctx) {
    ServeState *s = ctx->serve;
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->th.joinable()) s->th.join();
    cudaSetDevice(ctx->device);
    for (auto &sl : s->slots) cudaStreamSynchronize(sl->stream);
    for (auto &kv : s->reqs)
        if (kv.second.A) cudaFreeAsync(kv.second.A, s->slots[0]->stream);
    for (auto &sl : s->slots) {
        cudaStreamSynchronize(sl->stream);
        dyn_batch_free(sl->dyn);
        free_scratch(sl->plain);
        cudaStreamDestroy(sl->stream);
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    ctx->serve = nullptr;
}

static fe_status ensure_serve(fe_ctx *ctx) {
    if (ctx->serve) return FE_OK;
    cudaSetDevice(ctx->device);
    auto *s = new ServeState();
    s->ctx = ctx;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = ctx->device;
    cudaError_t e = cudaMemPoolCreate(&s->pool, &props);
    if (e != cudaSuccess) {
        delete s;
        return cuda_check(ctx, e, "cudaMemPoolCreate");
    }
    uint64_t keep = ~0ull;  // keep freed memory in the pool for reuse
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    for (int i = 0; i < ctx->serve_slots; ++i) {
        s->slots.emplace_back(new Slot());
        s->slots.back()->owner = s;
        cudaStreamCreateWithFlags(&s->slots.back()->stream, cudaStreamNonBlocking);
    }
    s->th = std::thread(scheduler, s);
    ctx->serve = s;
    return FE_OK;
}

}  // namespace fe

using namespace fe;

extern "C" {

}  // extern "C"

namespace {

// Validate one request and fill its record (everything but the ticket and the
// submission time). No lock held.
fe_status prepare_request(fe_ctx *ctx, const fe_request *req, Req &q) {
    MeshRec mesh;
    {
        std::lock_guard<std::mutex> lk(ctx->mesh_mu);
        auto it = ctx->meshes.find(req->mesh_id);
        if (it == ctx->meshes.end()) return set_error(ctx, FE_ERR_INVALID_ARG, "unknown mesh id");
        mesh = it->second;
    }
    if (req->coef_mode == FE_COEF_FUNCTION_U)
        return set_error(ctx, FE_ERR_UNSUPPORTED, "served requests take coefficient arrays");
    fe_elem_args a{};
    a.n_elem = mesh.n_elem;
    a.coords = mesh.coords;
    a.coords_layout = FE_LAYOUT_AOS;
    a.kind = req->kind;
    a.quad = req->quad;
    a.coef_mode = req->coef_mode;
    a.coefs = req->coefs;
    a.coefs_layout = FE_LAYOUT_AOS;
    a.prec = req->prec;
    fe_out o{};
    o.A = o.b = reinterpret_cast<void *>(uintptr_t(256));  // outputs are the context's
    o.layout = FE_LAYOUT_AOS;
    const fe_status st = fe_check_args(mesh.type, &a, &o);
    if (st != FE_OK) return set_error(ctx, st, fe_last_error(nullptr));
    const uint64_t ob = out_bytes_of(mesh, req->prec);
    if (ctx->hbm_used.load() + ob > ctx->hbm_budget)
        return set_error(ctx, FE_ERR_BUDGET, "request outputs can never fit the HBM budget");
    q.r = *req;
    q.mesh = mesh;
    q.out_bytes = ob;
    return FE_OK;
}

}  // namespace

extern "C" {

fe_status fe_serve_submit(fe_ctx *ctx, const fe_request *req, uint64_t *ticket) {
    if (!ctx || !req || !ticket) return set_error(ctx, FE_ERR_INVALID_ARG, "null argument");
    return fe_serve_submit_n(ctx, req, 1, ticket);
}

fe_status fe_serve_submit_n(fe_ctx *ctx, const fe_request *reqs, int n, uint64_t *tickets) {
    if (!ctx || n < 0 || (n > 0 && (!reqs || !tickets))) return set_error(ctx, FE_ERR_INVALID_ARG, "bad argument");
    if (n == 0) return FE_OK;
    std::vector<Req> recs(static_cast<size_t>(n));
    for (int i = 0; i < n; ++i) {
        const fe_status st = prepare_request(ctx, &reqs[i], recs[size_t(i)]);
        if (st != FE_OK) return st;  // nothing queued
    }
    fe_status st = ensure_serve(ctx);
    if (st != FE_OK) return st;
    ServeState *s = ctx->serve;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const double t = now_us();
        for (int i = 0; i < n; ++i) {
            const uint64_t tk = s->next_ticket++;
            Req &q = s->reqs[tk];
            q = recs[size_t(i)];
            q.t_submit = t;
            s->waiting.push_back(tk);
            tickets[i] = tk;
        }
    }
    s->cv.notify_all();
    return FE_OK;
}

fe_status fe_serve_cancel(fe_ctx *ctx, uint64_t ticket) {
    if (!ctx) return set_error(nullptr, FE_ERR_INVALID_ARG, "null context");
    ServeState *s = ctx->serve;
    if (!s) return set_error(ctx, FE_ERR_INVALID_ARG, "unknown ticket");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(ctx, FE_ERR_INVALID_ARG, "unknown ticket");
    if (it->second.state != 0) return set_error(ctx, FE_ERR_INVALID_ARG, "request already launched");
    auto w = std::find(s->waiting.begin(), s->waiting.end(), ticket);
    if (w != s->waiting.end()) s->waiting.erase(w);
    s->reqs.erase(it);   // admitted requests are launched under the same lock: nothing was reserved
    return FE_OK;
}

fe_status fe_serve_poll(fe_ctx *ctx, uint64_t ticket, fe_result *res) {
    if (!ctx || !res) return set_error(ctx, FE_ERR_INVALID_ARG, "null argument");
    ServeState *s = ctx->serve;
    if (!s) return set_error(ctx, FE_ERR_INVALID_ARG, "unknown ticket");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(ctx, FE_ERR_INVALID_ARG, "unknown ticket");
    Req &q = it->second;
    if (q.state == 1 && q.slot >= 0 && s->slots[q.slot]->done.load(std::memory_order_acquire)) reap(s);
    if (q.state != 2) return FE_NOT_READY;
    fill_result(q, res);
    return q.status == FE_OK ? FE_OK : q.status;
}

fe_status fe_serve_wait_any(fe_ctx *ctx, int64_t timeout_us, uint64_t *tickets, fe_result *results, int max,
                            int *n_out) {
    if (!ctx || !tickets || !results || !n_out || max <= 0 || timeout_us < 0)
        return set_error(ctx, FE_ERR_INVALID_ARG, "bad argument");
    *n_out = 0;
    fe_status st = ensure_serve(ctx);
    if (st != FE_OK) return st;
    ServeState *s = ctx->serve;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us);
    for (;;) {
        reap(s);
        int n = 0;
        while (n < max && !s->done_q.empty()) {
            const uint64_t tk = s->done_q.front();
            s->done_q.pop_front();
            auto it = s->reqs.find(tk);
            if (it == s->reqs.end() || it->second.returned) continue;  // released meanwhile
            it->second.returned = true;
            tickets[n] = tk;
            fill_result(it->second, &results[n]);
            ++n;
        }
        if (n > 0 || timeout_us == 0) {
            *n_out = n;
            return FE_OK;
        }
        // the slot callbacks wake the scheduler, whose reap wakes this wait; the
        // short period bounds the delay if a wake-up is missed
        if (s->done_cv.wait_until(lk, std::min(deadline, std::chrono::steady_clock::now() +
                                                             std::chrono::microseconds(500))) ==
                std::cv_status::timeout &&
            std::chrono::steady_clock::now() >= deadline) {
            reap(s);
            if (s->done_q.empty()) return FE_OK;
        }
    }
}

fe_status fe_serve_release(fe_ctx *ctx, uint64_t ticket) { return fe_serve_release_n(ctx, &ticket, 1); }

fe_status fe_serve_release_n(fe_ctx *ctx, const uint64_t *tickets, int n) {
    if (!ctx) return set_error(nullptr, FE_ERR_INVALID_ARG, "null context");
    if (n < 0 || (n > 0 && !tickets)) return set_error(ctx, FE_ERR_INVALID_ARG, "bad argument");
    if (n == 0) return FE_OK;
    ServeState *s = ctx->serve;
    if (!s) return set_error(ctx, FE_ERR_INVALID_ARG, "unknown ticket");
    std::vector<std::pair<void *, cudaStream_t>> frees;
    frees.reserve(size_t(n));
    {
        std::lock_guard<std::mutex> lk(s->mu);
        // all or nothing: every ticket must be known, finished and listed once
        for (int i = 0; i < n; ++i) {
            auto it = s->reqs.find(tickets[i]);
            if (it == s->reqs.end()) return set_error(ctx, FE_ERR_INVALID_ARG, "unknown ticket");
            if (it->second.state != 2) return set_error(ctx, FE_ERR_INVALID_ARG, "request still running");
            for (int j = 0; j < i; ++j)
                if (tickets[j] == tickets[i]) return set_error(ctx, FE_ERR_INVALID_ARG, "ticket listed twice");
        }
        for (int i = 0; i < n; ++i) {
            auto it = s->reqs.find(tickets[i]);
            Req &q = it->second;
            // the one allocation that also holds b and the flags
            frees.emplace_back(q.A, s->slots[std::max(q.slot, 0)]->stream);
            s->out_used -= q.out_bytes;
            s->reqs.erase(it);
        }
    }
    s->cv.notify_all();
    // stream-ordered frees outside the lock
    cudaSetDevice(ctx->device);
    for (auto &f : frees)
        if (f.first) cudaFreeAsync(f.first, f.second);
    return FE_OK;
}

}  // extern "C"
