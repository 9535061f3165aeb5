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
// elements (the first request always fits).
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
};

struct ServeState;

constexpr uint64_t kFeedElems = uint64_t(16) << 20;    // ~1 ms of GPU work in flight
constexpr uint64_t kLaunchElems = uint64_t(64) << 20;
struct Slot {
    ServeState *owner = nullptr;
    cudaStream_t stream = nullptr;
    bool busy = false;                 // guarded by the state's mutex
    std::atomic<int> done{0};          // set by the stream's host callback
    double t_done = 0;                 // written by the callback before `done`
    std::vector<uint64_t> tickets;
    uint64_t elems = 0;                // elements of the launch in flight (mutex)
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

// Mark the requests of finished slots done and free the slots (lock held).
static void reap(ServeState *s) {
    for (auto &up : s->slots) {
        Slot &sl = *up;
        if (!sl.busy || !sl.done.load(std::memory_order_acquire)) continue;
        for (uint64_t tk : sl.tickets) {
            auto it = s->reqs.find(tk);
            if (it != s->reqs.end()) {
                it->second.t_done = sl.t_done;
                it->second.state = 2;
            }
        }
        sl.tickets.clear();
        sl.elems = 0;
        sl.done.store(0, std::memory_order_relaxed);
        sl.busy = false;
    }
}

static uint64_t out_bytes_of(const MeshRec &m, fe_precision prec) {
    const uint64_t ns = uint64_t(ns_of(m.type)), cs = prec == FE_FP32_MIXED ? 4 : 8;
    auto r256 = [](uint64_t v) { return (v + 255) / 256 * 256; };
    return r256(uint64_t(m.n_elem) * ns * ns * cs) + r256(uint64_t(m.n_elem) * ns * cs) + r256(uint64_t(m.n_elem));
}

// Launch everything admitted into a free slot (called with the lock held).
static void launch_slot(ServeState *s, int si, std::vector<uint64_t> &batch) {
    fe_ctx *ctx = s->ctx;
    Slot &sl = *s->slots[si];
    sl.busy = true;
    sl.tickets = batch;
    sl.elems = 0;
    for (uint64_t tk : batch) sl.elems += uint64_t(s->reqs[tk].mesh.n_elem);
    std::vector<BatchItemDev> items;
    const double t = now_us();
    fe_status st = FE_OK;
    for (uint64_t tk : batch) {
        Req &q = s->reqs[tk];
        q.t_launch = t;
        q.state = 1;
        q.slot = si;
        const MeshRec &m = q.mesh;
        // outputs from the context's stream-ordered pool
        const uint64_t ns = ns_of(m.type), cs = q.r.prec == FE_FP32_MIXED ? 4 : 8;
        const uint64_t bA = uint64_t(m.n_elem) * ns * ns * cs, bB = uint64_t(m.n_elem) * ns * cs;
        cudaError_t e = cudaMallocFromPoolAsync(&q.A, bA, s->pool, sl.stream);
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&q.b, bB, s->pool, sl.stream);
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&q.flags), size_t(m.n_elem), s->pool, sl.stream);
        if (e != cudaSuccess) {
            q.status = cuda_check(ctx, e, "cudaMallocFromPoolAsync(serve outputs)");
            continue;
        }
        fe_elem_args a{};
        a.n_elem = m.n_elem;
        a.coords = m.coords;
        a.coords_layout = FE_LAYOUT_AOS;
        a.kind = q.r.kind;
        a.quad = q.r.quad;
        a.coef_mode = q.r.coef_mode;
        a.coefs = q.r.coefs;
        a.coefs_layout = FE_LAYOUT_AOS;
        a.prec = q.r.prec;
        a.memory = FE_MEM_DEVICE;
        fe_out o{};
        o.A = q.A;
        o.b = q.b;
        o.layout = FE_LAYOUT_AOS;
        o.flags = q.flags;
        o.memory = FE_MEM_DEVICE;
        if (q.r.prec == FE_FP32_MIXED) {
            BatchItemDev d;
            memset(&d, 0, sizeof d);
            d.p.n = m.n_elem;
            d.p.X = m.coords;
            d.p.xs = m.n_elem;
            d.p.C = q.r.coefs;
            d.p.cs = m.n_elem;
            d.p.A = q.A;
            d.p.B = q.b;
            d.p.os = m.n_elem;
            d.p.flags = q.flags;
            d.p.item = unsigned(items.size());
            d.combo = batch_combo(m.type, q.r.kind, q.r.quad, q.r.coef_mode == FE_COEF_PER_QPOINT);
            items.push_back(d);
        } else {
            const Shape sh = default_shape(m.type);
            q.status = launch_set(ctx, m.type, &a, &o, sl.plain, sl.stream, &sh);
        }
    }
    if (!items.empty()) {
        st = dyn_batch_launch(ctx, sl.dyn, items, sl.stream);
        if (st != FE_OK)
            for (uint64_t tk : batch) {
                Req &q = s->reqs[tk];
                if (q.r.prec == FE_FP32_MIXED) q.status = st;
            }
    }
    cudaLaunchHostFunc(sl.stream, on_slot_done, &sl);
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
                launch_slot(s, free_slot, batch);
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
    for (auto &kv : s->reqs) {
        if (kv.second.A) cudaFreeAsync(kv.second.A, s->slots[0]->stream);
        if (kv.second.b) cudaFreeAsync(kv.second.b, s->slots[0]->stream);
        if (kv.second.flags) cudaFreeAsync(kv.second.flags, s->slots[0]->stream);
    }
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

fe_status fe_serve_submit(fe_ctx *ctx, const fe_request *req, uint64_t *ticket) {
    if (!ctx || !req || !ticket) return set_error(ctx, FE_ERR_INVALID_ARG, "null argument");
    MeshRec mesh;
    {
        std::lock_guard<std::mutex> lk(ctx->mesh_mu);
        auto it = ctx->meshes.find(req->mesh_id);
        if (it == ctx->meshes.end()) return set_error(ctx, FE_ERR_INVALID_ARG, "unknown mesh id");
        mesh = it->second;
    }
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
    fe_status st = fe_check_args(mesh.type, &a, &o);
    if (st != FE_OK) return set_error(ctx, st, fe_last_error(nullptr));
    const uint64_t ob = out_bytes_of(mesh, req->prec);
    if (ctx->hbm_used.load() + ob > ctx->hbm_budget)
        return set_error(ctx, FE_ERR_BUDGET, "request outputs can never fit the HBM budget");
    st = ensure_serve(ctx);
    if (st != FE_OK) return st;
    ServeState *s = ctx->serve;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const uint64_t tk = s->next_ticket++;
        Req &q = s->reqs[tk];
        q.r = *req;
        q.mesh = mesh;
        q.out_bytes = ob;
        q.t_submit = now_us();
        s->waiting.push_back(tk);
        *ticket = tk;
    }
    s->cv.notify_all();
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
    res->status = q.status;
    res->type = q.mesh.type;
    res->n_elem = q.mesh.n_elem;
    res->A = q.A;
    res->b = q.b;
    res->flags = q.flags;
    res->t_submit_us = q.t_submit;
    res->t_launch_us = q.t_launch;
    res->t_done_us = q.t_done;
    return q.status == FE_OK ? FE_OK : q.status;
}

fe_status fe_serve_release(fe_ctx *ctx, uint64_t ticket) {
    if (!ctx) return set_error(nullptr, FE_ERR_INVALID_ARG, "null context");
    ServeState *s = ctx->serve;
    if (!s) return set_error(ctx, FE_ERR_INVALID_ARG, "unknown ticket");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return set_error(ctx, FE_ERR_INVALID_ARG, "unknown ticket");
        Req &q = it->second;
        if (q.state != 2) return set_error(ctx, FE_ERR_INVALID_ARG, "request still running");
        cudaSetDevice(ctx->device);
        cudaStream_t st = s->slots[std::max(q.slot, 0)]->stream;
        if (q.A) cudaFreeAsync(q.A, st);
        if (q.b) cudaFreeAsync(q.b, st);
        if (q.flags) cudaFreeAsync(q.flags, st);
        s->out_used -= q.out_bytes;
        s->reqs.erase(it);
    }
    s->cv.notify_all();
    return FE_OK;
}

}  // extern "C"
