// Resident meshes and batched integration (host side): tile plans, the
// autotuner of the batched launch, and CUDA-graph capture of
// {counter reset, one persistent kernel per combination on parallel branches,
// fix-up kernel}.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <functional>
#include <list>
#include <string>

#include "fe_runtime.h"

namespace fe {

// ---------------------------------------------------------------------------
// Element-contiguous copy of plane-major coordinates (resident meshes).
// ---------------------------------------------------------------------------
__global__ void soa_to_aos_kernel(const double *__restrict__ in, int64_t stride, int nx, int64_t n,
                                  double *__restrict__ out) {
    const int64_t total = n * nx;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t e = i / nx;
        const int j = int(i - e * nx);
        out[i] = in[j * stride + e];
    }
}

// One persistent launch per combination present: its items are a contiguous
// run of the plan's segment table, its tiles numbered 0..n_tiles-1, with its own
// counter.
struct ClassLaunch {
    int combo = 0;
    int block = 128;                 // elements per tile of this combination
    int persistent = 1;              // 1: counter-driven persistent grid; 0: one block per tile
    unsigned seg_off = 0, n_segs = 0, n_tiles = 0;
    int grid = 0;
    int64_t smem = 0;
};

struct BatchPlan {
    size_t key = 0;
    std::vector<unsigned char> items_bytes;
    int pinned_block = 0, pinned_tpe = 1, pinned_pers = 1;   // the pinned shape it was built with (block 0: none)
    BatchItemDev *d_items = nullptr;
    BatchSeg *d_segs = nullptr;
    unsigned n_items = 0, n_segs = 0;
    unsigned *d_counter = nullptr;   // kCombos counters
    Scratch scratch;
    std::vector<ClassLaunch> classes;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

struct BatchCache {
    std::list<BatchPlan *> plans;  // most recent first
    cudaStream_t capture_stream = nullptr;
    // parallel branches of one step: a stream per combination, fork and join events
    cudaStream_t branch[kCombos] = {nullptr};
    cudaEvent_t ev_fork = nullptr, ev_join[kCombos] = {nullptr};
};

static void free_plan(BatchPlan *pl) {
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->d_items) cudaFree(pl->d_items);
    if (pl->d_segs) cudaFree(pl->d_segs);
    if (pl->d_counter) cudaFree(pl->d_counter);
    free_scratch(pl->scratch);
    delete pl;
}

void batch_destroy(fe_ctx *ctx) {
    if (!ctx->batch) return;
    for (auto *pl : ctx->batch->plans) free_plan(pl);
    if (ctx->batch->capture_stream) cudaStreamDestroy(ctx->batch->capture_stream);
    for (int i = 0; i < kCombos; ++i) {
        if (ctx->batch->branch[i]) cudaStreamDestroy(ctx->batch->branch[i]);
        if (ctx->batch->ev_join[i]) cudaEventDestroy(ctx->batch->ev_join[i]);
    }
    if (ctx->batch->ev_fork) cudaEventDestroy(ctx->batch->ev_fork);
    delete ctx->batch;
    ctx->batch = nullptr;
}

// Relative cost of one element of a combination (bytes moved plus arithmetic),
// used only to launch the heaviest combinations first.
static double combo_cost(int combo) {
    static const double cost[12] = {1.0, 1.0, 1.1, 1.2, 1.4, 1.5, 1.5, 1.8, 2.5, 2.6, 6.0, 8.0};
    if (combo >= 12 && combo < kCombos) combo -= 4;   // the same prisms, two threads each
    return combo >= 0 && combo < 12 ? cost[combo] : 1.0;
}

// Segment table of tiles of Bc[combination] consecutive elements: items grouped
// by combination (heaviest combination first) and, within one, largest first,
// each with the index of its first tile. Work is proportional to the number of
// items, not of tiles. Fails if a combination has 2^32 tiles or more.
static bool make_segs(const std::vector<BatchItemDev> &items, const int *Bc, const int *Pc, std::vector<BatchSeg> &out,
                      std::vector<ClassLaunch> &classes) {
    std::vector<std::vector<unsigned>> per(kCombos);
    for (unsigned i = 0; i < items.size(); ++i) {
        const int c = items[i].combo;
        if (c >= 0 && c < kCombos && items[i].p.n > 0) per[c].push_back(i);
    }
    std::vector<int> order(kCombos);
    for (int c = 0; c < kCombos; ++c) order[c] = c;
    std::stable_sort(order.begin(), order.end(), [](int a, int b) { return combo_cost(a) > combo_cost(b); });
    out.clear();
    classes.clear();
    for (int c : order) {
        if (per[c].empty()) continue;
        std::stable_sort(per[c].begin(), per[c].end(),
                         [&](unsigned a, unsigned b) { return items[a].p.n > items[b].p.n; });
        ClassLaunch cl;
        cl.combo = c;
        cl.block = Bc[c];
        cl.persistent = Pc[c];
        const int B = cl.block;
        cl.seg_off = unsigned(out.size());
        cl.n_segs = unsigned(per[c].size());
        uint64_t tiles = 0;
        for (unsigned i : per[c]) {
            out.push_back(BatchSeg{i, unsigned(tiles), static_cast<long long>(items[i].p.n)});
            tiles += uint64_t((items[i].p.n + B - 1) / B);
            if (tiles >= (uint64_t(1) << 32)) return false;
        }
        cl.n_tiles = unsigned(tiles);
        classes.push_back(cl);
    }
    return true;
}

static std::mutex g_attr_mu;
static int64_t g_attr_set[kCombos] = {0};

// Shared memory attribute and grid of each class launch: SMs x resident blocks
// (persistent) or one block per tile.
static fe_status size_classes(fe_ctx *ctx, std::vector<ClassLaunch> &classes) {
    for (auto &cl : classes) {
        const int B = cl.block;
        const void *k = kernel_batch(cl.combo);
        const int threads = B * batch_tpe(cl.combo);
        if (threads > 256) return set_error(ctx, FE_ERR_UNSUPPORTED, "batched tile of more than 256 threads");
        cl.smem = batch_smem_bytes(cl.combo, B);
        if (cl.smem + 1024 > ctx->max_smem_optin)
            return set_error(ctx, FE_ERR_UNSUPPORTED, "batched tile does not fit in shared memory");
        {
            std::lock_guard<std::mutex> lk(g_attr_mu);
            if (cl.smem > g_attr_set[cl.combo]) {
                fe_status st = cuda_check(ctx, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(cl.smem)),
                                          "cudaFuncSetAttribute(batch)");
                if (st != FE_OK) return st;
                g_attr_set[cl.combo] = cl.smem;
            }
        }
        // resident blocks per SM for (combination, B), queried once per process
        static std::mutex occ_mu;
        static std::map<std::pair<int, int>, int> occ;
        int per_sm = 0;
        {
            std::lock_guard<std::mutex> lk(occ_mu);
            auto it = occ.find({cl.combo, B});
            if (it != occ.end()) {
                per_sm = it->second;
            } else {
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, size_t(cl.smem));
                occ[{cl.combo, B}] = per_sm;
            }
        }
        cl.grid = int(std::min<int64_t>(cl.persistent ? int64_t(std::max(1, per_sm)) * ctx->sms : int64_t(0x7FFFFFFF),
                                        cl.n_tiles));
    }
    return FE_OK;
}

static fe_status upload_segs(fe_ctx *ctx, BatchPlan *pl, const std::vector<BatchItemDev> &items, const int *Bc,
                             const int *Pc) {
    std::vector<BatchSeg> segs;
    if (!make_segs(items, Bc, Pc, segs, pl->classes))
        return set_error(ctx, FE_ERR_UNSUPPORTED, "2^32 or more tiles of one combination in a batch");
    if (pl->d_segs) cudaFree(pl->d_segs);
    pl->d_segs = nullptr;
    pl->n_segs = unsigned(segs.size());
    fe_status st = ctx_malloc(ctx, reinterpret_cast<void **>(&pl->d_segs),
                              std::max<size_t>(1, segs.size()) * sizeof(BatchSeg), "cudaMalloc(segments)");
    if (st != FE_OK) return st;
    st = cuda_check(ctx, cudaMemcpy(pl->d_segs, segs.data(), segs.size() * sizeof(BatchSeg), cudaMemcpyHostToDevice),
                    "cudaMemcpy(segments)");
    if (st != FE_OK) return st;
    return size_classes(ctx, pl->classes);
}

// Streams and events of the parallel branches (created once per context).
static fe_status ensure_branches(fe_ctx *ctx, size_t n) {
    BatchCache *bc = ctx->batch;
    cudaError_t e = cudaSuccess;
    if (!bc->ev_fork) e = cudaEventCreateWithFlags(&bc->ev_fork, cudaEventDisableTiming);
    for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
        if (!bc->branch[i]) e = cudaStreamCreateWithFlags(&bc->branch[i], cudaStreamNonBlocking);
        if (e == cudaSuccess && !bc->ev_join[i]) e = cudaEventCreateWithFlags(&bc->ev_join[i], cudaEventDisableTiming);
    }
    return cuda_check(ctx, e, "batch branch streams");
}

// The kernel of one combination on stream `s`; with `reset`, its tile counter and
// the fix-up count are zeroed first (the combination run alone, when tuning).
static fe_status launch_class(fe_ctx *ctx, BatchPlan *pl, const ClassLaunch &cl, cudaStream_t s, bool reset) {
    cudaError_t e = cudaSuccess;
    if (reset) {
        e = cudaMemsetAsync(pl->d_counter + cl.combo, 0, sizeof(unsigned), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(pl->scratch.fix_count, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return cuda_check(ctx, e, "cudaMemsetAsync(batch class)");
    }
    int *status = ctx->scratch.status;
    const BatchSeg *segs = pl->d_segs + cl.seg_off;
    unsigned n_segs = cl.n_segs, n_tiles = cl.n_tiles;
    unsigned *counter = cl.persistent ? pl->d_counter + cl.combo : nullptr;
    void *args[] = {&pl->d_items, &pl->n_items, &segs, &n_segs, &n_tiles, &counter, &status};
    e = cudaLaunchKernel(kernel_batch(cl.combo), dim3(cl.grid), dim3(cl.block * batch_tpe(cl.combo)), args,
                         size_t(cl.smem), s);
    return cuda_check(ctx, e, "cudaLaunchKernel(batch)");
}

// Enqueue {counter reset, one persistent kernel per combination, fix-up kernel}.
// With `branches`, the combinations' kernels go on parallel branches (a fork
// from `st`, one stream each, a join back before the fix-up), so that the blocks
// of the next combinations fill the SMs that a finishing one leaves idle instead
// of waiting for its last tiles; captured, they become parallel graph branches.
static fe_status enqueue_batch(fe_ctx *ctx, BatchPlan *pl, cudaStream_t st, bool counters_zeroed = false,
                               bool branches = false) {
    cudaError_t e = cudaSuccess;
    if (!counters_zeroed) {
        e = cudaMemsetAsync(pl->d_counter, 0, kCombos * sizeof(unsigned), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(pl->scratch.fix_count, 0, sizeof(unsigned), st);
        if (e != cudaSuccess) return cuda_check(ctx, e, "cudaMemsetAsync(batch)");
    }
    int *status = ctx->scratch.status;
    const bool fork = branches && pl->classes.size() > 1;
    BatchCache *bc = ctx->batch;
    if (fork) {
        fe_status fs = ensure_branches(ctx, pl->classes.size());
        if (fs != FE_OK) return fs;
        e = cudaEventRecord(bc->ev_fork, st);
        if (e != cudaSuccess) return cuda_check(ctx, e, "cudaEventRecord(batch fork)");
    }
    for (size_t i = 0; i < pl->classes.size(); ++i) {
        const auto &cl = pl->classes[i];
        cudaStream_t ls = fork ? bc->branch[i] : st;
        if (fork) {
            e = cudaStreamWaitEvent(ls, bc->ev_fork, 0);
            if (e != cudaSuccess) return cuda_check(ctx, e, "cudaStreamWaitEvent(batch fork)");
        }
        fe_status ls_st = launch_class(ctx, pl, cl, ls, false);
        if (ls_st != FE_OK) return ls_st;
        if (fork) {
            e = cudaEventRecord(bc->ev_join[i], ls);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, bc->ev_join[i], 0);
            if (e != cudaSuccess) return cuda_check(ctx, e, "batch join");
        }
    }
    unsigned long long *list = pl->scratch.fix_list;
    unsigned *count = pl->scratch.fix_count;
    unsigned cap = pl->scratch.fix_cap;
    void *fargs[] = {&pl->d_items, &pl->n_items, &list, &count, &cap, &status};
    e = cudaLaunchKernel(kernel_batch_fixup(), dim3(ctx->sms * 4), dim3(256), fargs, 0, st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "cudaLaunchKernel(batch fix-up)");
    return FE_OK;
}

static int plan_launches(const BatchPlan *pl) { return int(pl->classes.size()) + 1; }

static fe_status build_plan(fe_ctx *ctx, const fe_batch_item *items, int n, size_t key, BatchPlan *&out) {
    auto *pl = new BatchPlan();
    pl->key = key;
    pl->pinned_block = ctx->batch_shape.block;
    pl->pinned_tpe = ctx->batch_shape.tpe;
    pl->pinned_pers = ctx->batch_shape.persistent;
    pl->items_bytes.assign(reinterpret_cast<const unsigned char *>(items),
                           reinterpret_cast<const unsigned char *>(items) + sizeof(fe_batch_item) * n);
    std::vector<BatchItemDev> dev(n);
    uint64_t total = 0;
    for (int i = 0; i < n; ++i) total += uint64_t(items[i].args.n_elem);
    fe_status st = ensure_scratch(ctx, pl->scratch, total);
    if (st == FE_OK) st = ctx_malloc(ctx, reinterpret_cast<void **>(&pl->d_counter), 256, "cudaMalloc(counter)");
    for (int i = 0; i < n && st == FE_OK; ++i) {
        const fe_elem_args &a = items[i].args;
        const fe_out &o = items[i].out;
        BatchItemDev &d = dev[i];
        memset(&d, 0, sizeof d);
        d.p.n = a.n_elem;
        d.p.X = a.coords;
        d.p.xs = a.n_elem;
        d.p.C = a.coefs;
        d.p.cs = a.n_elem;
        d.p.A = o.A;
        d.p.B = o.b;
        d.p.os = a.n_elem;
        d.p.flags = o.flags;
        d.p.fix_list = pl->scratch.fix_list;
        d.p.fix_count = pl->scratch.fix_count;
        d.p.fix_cap = pl->scratch.fix_cap;
        d.p.item = unsigned(i);
        d.p.status = ctx->scratch.status;
        d.combo = batch_combo(items[i].type, a.kind, a.quad, a.coef_mode == FE_COEF_PER_QPOINT);
    }
    if (st == FE_OK) {
        pl->n_items = unsigned(n);
        st = ctx_malloc(ctx, reinterpret_cast<void **>(&pl->d_items), sizeof(BatchItemDev) * n, "cudaMalloc(items)");
    }
    if (st == FE_OK)
        st = cuda_check(ctx, cudaMemcpy(pl->d_items, dev.data(), sizeof(BatchItemDev) * n, cudaMemcpyHostToDevice),
                        "cudaMemcpy(items)");
    if (!ctx->batch->capture_stream) cudaStreamCreateWithFlags(&ctx->batch->capture_stream, cudaStreamNonBlocking);
    cudaStream_t cs = ctx->batch->capture_stream;
    // launch shape of each combination: elements per tile, persistent or one block
    // per tile and, for prisms, one or two threads per element; tuned per
    // combination (each timed alone), pinned, or 128 / persistent / one
    bool any_prism = false;
    for (const auto &d : dev) any_prism = any_prism || (d.combo >= 8 && d.combo < 12);
    auto base_of = [](int c) { return c >= 12 ? c - 4 : c; };   // the one-thread combination of a pair one
    int Bb[kCombos], Tb[kCombos], Pb[kCombos];                  // per base combination
    for (int c = 0; c < kCombos; ++c) Bb[c] = 128, Tb[c] = 1, Pb[c] = 1;
    auto set_tpe = [&](const int *T) -> fe_status {
        for (auto &d : dev)
            if (d.combo >= 8) {
                const int b = base_of(d.combo);
                d.combo = T[b] == 2 ? batch_pair_combo(b) : b;
            }
        return cuda_check(ctx, cudaMemcpy(pl->d_items, dev.data(), sizeof(BatchItemDev) * n, cudaMemcpyHostToDevice),
                          "cudaMemcpy(items)");
    };
    auto upload = [&](const int *B, const int *P) -> fe_status {
        int Bf[kCombos], Pf[kCombos];
        for (int c = 0; c < kCombos; ++c) Bf[c] = B[base_of(c)], Pf[c] = P[base_of(c)];
        return upload_segs(ctx, pl, dev, Bf, Pf);
    };
    if (ctx->batch_shape.block > 0) {            // pinned by fe_batch_set_shape
        for (int c = 0; c < kCombos; ++c)
            Bb[c] = ctx->batch_shape.block, Tb[c] = ctx->batch_shape.tpe, Pb[c] = ctx->batch_shape.persistent;
    } else if (st == FE_OK && ctx->autotune) {
        float best[kCombos];
        for (int c = 0; c < kCombos; ++c) best[c] = 1e30f;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int tpe = 1; tpe <= (any_prism ? 2 : 1) && st == FE_OK; ++tpe)
            for (int pers = 1; pers >= 0 && st == FE_OK; --pers)
                for (int B : {64, 128, 256}) {
                    int Bt[kCombos], Tt[kCombos], Pt[kCombos];
                    for (int c = 0; c < kCombos; ++c) Bt[c] = B, Tt[c] = tpe, Pt[c] = pers;
                    st = set_tpe(Tt);
                    if (st == FE_OK) st = upload(Bt, Pt);
                    if (st == FE_ERR_UNSUPPORTED) {   // tile too large for shared memory or threads
                        st = FE_OK;
                        continue;
                    }
                    if (st != FE_OK) break;
                    // each combination alone: counter and fix-up count reset, then its kernel
                    for (const auto &cl : pl->classes) {
                        float t = 0.0f;
                        for (int r = 0; r < 4 && st == FE_OK; ++r) {   // one warm-up, three timed
                            if (r == 1) cudaEventRecord(e0, cs);
                            st = launch_class(ctx, pl, cl, cs, true);
                        }
                        cudaEventRecord(e1, cs);
                        if (st != FE_OK) break;
                        cudaError_t ce = cudaEventSynchronize(e1);
                        if (ce != cudaSuccess) {
                            st = cuda_check(ctx, ce, "batch tuning");
                            break;
                        }
                        cudaEventElapsedTime(&t, e0, e1);
                        const int b = base_of(cl.combo);
                        if (t < best[b]) {
                            best[b] = t;
                            Bb[b] = B;
                            Tb[b] = tpe;
                            Pb[b] = pers;
                        }
                    }
                }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    if (st == FE_OK) st = set_tpe(Tb);
    if (st == FE_OK) st = upload(Bb, Pb);
    // capture the launch sequence once; later submissions replay it
    if (st == FE_OK) {
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) st = cuda_check(ctx, e, "cudaStreamBeginCapture");
        if (st == FE_OK) {
            fe_status est = enqueue_batch(ctx, pl, cs, false, true);
            e = cudaStreamEndCapture(cs, &pl->graph);
            if (est != FE_OK) st = est;
            else if (e != cudaSuccess) st = cuda_check(ctx, e, "cudaStreamEndCapture");
        }
        if (st == FE_OK) st = cuda_check(ctx, cudaGraphInstantiate(&pl->exec, pl->graph, 0), "cudaGraphInstantiate");
    }
    if (st != FE_OK) {
        free_plan(pl);
        return st;
    }
    out = pl;
    return FE_OK;
}

// ---------------------------------------------------------------------------
// Dynamically built batch (serving).
// ---------------------------------------------------------------------------
void dyn_batch_free(DynBatch &db) {
    if (db.d_tab) cudaFree(db.d_tab);
    if (db.h_tab) cudaFreeHost(db.h_tab);
    free_scratch(db.scratch);
    db = DynBatch{};
}

// The caller guarantees that the previous launch on this DynBatch has finished
// (its pinned staging and device table are reused).
fe_status dyn_batch_launch(fe_ctx *ctx, DynBatch &db, std::vector<BatchItemDev> &items, cudaStream_t st) {
    // tiles of 128 tetrahedra and 64 prisms, one thread per element: the shapes the
    // batch autotuner keeps for these combinations on the 256-mesh workload (a
    // served launch is not tuned: it is built per launch)
    constexpr size_t kCountersOff = 0, kFixCountOff = 64, kItemsOff = 128;
    uint64_t total = 0;
    for (auto &it : items) total += uint64_t(it.p.n);
    // The fix-up list and the tables grow geometrically (the list from 4M elements):
    // a growth frees the old buffer, and cudaFree waits for the whole device, so a
    // serving loop should meet only a few of them, early.
    uint64_t want = total;
    if (want > db.scratch.fix_cap)
        want = std::min<uint64_t>(std::max<uint64_t>({want, 2 * uint64_t(db.scratch.fix_cap), uint64_t(1) << 22}),
                                  0xFFFFFFFFull);
    fe_status r = ensure_scratch(ctx, db.scratch, std::max(want, total));
    if (r != FE_OK) return r;
    std::vector<ClassLaunch> classes;
    std::vector<BatchSeg> segs;
    int Bc[kCombos], Pc[kCombos];
    for (int c = 0; c < kCombos; ++c) Bc[c] = c >= 8 ? 64 : 128, Pc[c] = 1;
    if (!make_segs(items, Bc, Pc, segs, classes))
        return set_error(ctx, FE_ERR_UNSUPPORTED, "2^32 or more tiles of one combination in a batch");
    const size_t items_bytes = (items.size() * sizeof(BatchItemDev) + 15) / 16 * 16;
    const size_t segs_off = kItemsOff + items_bytes;
    const size_t need = segs_off + std::max<size_t>(segs.size(), 1) * sizeof(BatchSeg);
    if (need > db.cap_tab) {
        const size_t cap = std::max({need, 2 * db.cap_tab, size_t(64) << 10});
        if (db.d_tab) cudaFree(db.d_tab);
        if (db.h_tab) cudaFreeHost(db.h_tab);
        db.d_tab = db.h_tab = nullptr;
        db.cap_tab = 0;
        r = ctx_malloc(ctx, reinterpret_cast<void **>(&db.d_tab), cap, "cudaMalloc(batch table)");
        if (r == FE_OK) r = cuda_check(ctx, cudaMallocHost(&db.h_tab, cap), "cudaMallocHost(batch table)");
        if (r != FE_OK) return r;
        db.cap_tab = cap;
    }
    unsigned *d_fix_count = reinterpret_cast<unsigned *>(db.d_tab + kFixCountOff);
    for (auto &it : items) {
        it.p.fix_list = db.scratch.fix_list;
        it.p.fix_count = d_fix_count;
        it.p.fix_cap = db.scratch.fix_cap;
        it.p.status = ctx->scratch.status;
    }
    memset(db.h_tab, 0, kItemsOff);
    memcpy(db.h_tab + kItemsOff, items.data(), items.size() * sizeof(BatchItemDev));
    memcpy(db.h_tab + segs_off, segs.data(), segs.size() * sizeof(BatchSeg));
    cudaError_t e = cudaMemcpyAsync(db.d_tab, db.h_tab, segs_off + segs.size() * sizeof(BatchSeg), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "cudaMemcpyAsync(batch table)");
    r = size_classes(ctx, classes);
    if (r != FE_OK) return r;
    BatchPlan pl;
    pl.d_items = reinterpret_cast<BatchItemDev *>(db.d_tab + kItemsOff);
    pl.d_segs = reinterpret_cast<BatchSeg *>(db.d_tab + segs_off);
    pl.n_items = unsigned(items.size());
    pl.n_segs = unsigned(segs.size());
    pl.d_counter = reinterpret_cast<unsigned *>(db.d_tab + kCountersOff);
    pl.scratch = db.scratch;
    pl.scratch.fix_count = d_fix_count;
    pl.classes = classes;
    r = enqueue_batch(ctx, &pl, st, true);
    // the plan only borrowed the tables
    pl.d_items = nullptr;
    pl.d_segs = nullptr;
    pl.d_counter = nullptr;
    pl.scratch = Scratch{};
    if (r == FE_OK) g_launches.fetch_add(uint64_t(plan_launches(&pl)));
    return r;
}

}  // namespace fe

using namespace fe;

extern "C" {

fe_status fe_mesh_register(fe_ctx *ctx, fe_elem_type type, int64_t n_elem, const double *coords, fe_layout layout,
                           fe_memory memory, int64_t *mesh_id) {
    if (!ctx || !mesh_id) return set_error(ctx, FE_ERR_INVALID_ARG, "null argument");
    if ((type != FE_TET && type != FE_PRISM) || n_elem <= 0 || !coords)
        return set_error(ctx, FE_ERR_INVALID_ARG, "bad mesh description");
    if ((layout != FE_LAYOUT_SOA && layout != FE_LAYOUT_AOS) || (memory != FE_MEM_DEVICE && memory != FE_MEM_HOST))
        return set_error(ctx, FE_ERR_INVALID_ARG, "bad layout or memory kind");
    cudaSetDevice(ctx->device);
    const int nx = 3 * ns_of(type);
    const uint64_t bytes = uint64_t(n_elem) * nx * 8;
    if (ctx->hbm_used.load() + bytes > ctx->hbm_budget)
        return set_error(ctx, FE_ERR_BUDGET, "resident mesh does not fit the HBM budget");
    double *d = nullptr;
    fe_status st = ctx_malloc(ctx, reinterpret_cast<void **>(&d), bytes, "cudaMalloc(mesh)");
    if (st != FE_OK) return st;
    cudaError_t e = cudaSuccess;
    if (layout == FE_LAYOUT_AOS) {
        e = cudaMemcpy(d, coords, bytes, memory == FE_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice);
    } else {
        const double *src = coords;
        double *tmp = nullptr;
        if (memory == FE_MEM_HOST) {
            e = cudaMalloc(&tmp, bytes);
            if (e == cudaSuccess) e = cudaMemcpy(tmp, coords, bytes, cudaMemcpyHostToDevice);
            src = tmp;
        }
        if (e == cudaSuccess) {
            const int64_t total = n_elem * nx;
            const int grid = int(std::min<int64_t>((total + 255) / 256, int64_t(ctx->sms) * 8));
            soa_to_aos_kernel<<<grid, 256>>>(src, n_elem, nx, n_elem, d);
            g_launches.fetch_add(1);
            e = cudaDeviceSynchronize();
        }
        if (tmp) cudaFree(tmp);
    }
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_check(ctx, e, "mesh upload");
    }
    std::lock_guard<std::mutex> lk(ctx->mesh_mu);
    const int64_t id = ctx->next_mesh++;
    ctx->meshes[id] = MeshRec{type, n_elem, d, bytes};
    ctx->hbm_used += bytes;
    *mesh_id = id;
    return FE_OK;
}

fe_status fe_mesh_release(fe_ctx *ctx, int64_t mesh_id) {
    if (!ctx) return set_error(nullptr, FE_ERR_INVALID_ARG, "null context");
    std::lock_guard<std::mutex> lk(ctx->mesh_mu);
    auto it = ctx->meshes.find(mesh_id);
    if (it == ctx->meshes.end()) return set_error(ctx, FE_ERR_INVALID_ARG, "unknown mesh id");
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    cudaFree(it->second.coords);
    ctx->hbm_used -= it->second.bytes;
    ctx->meshes.erase(it);
    return FE_OK;
}

fe_status fe_batch_set_shape(fe_ctx *ctx, const fe_launch_shape *shape) {
    if (!ctx) return set_error(nullptr, FE_ERR_INVALID_ARG, "null context");
    if (!shape) {
        ctx->batch_shape = Shape{0, 1, 1};
        return FE_OK;
    }
    const int B = shape->elems_per_block, t = shape->threads_per_elem;
    if ((t != 1 && t != 2) || B < 32 || B % 32 || B * t > 256 || (shape->persistent != 0 && shape->persistent != 1))
        return set_error(ctx, FE_ERR_INVALID_ARG, "bad batched launch shape");
    ctx->batch_shape = Shape{B, shape->persistent, t};
    return FE_OK;
}

fe_status fe_batch_submit(fe_ctx *ctx, const fe_batch_item *items, int n_items, void *stream) {
    TraceRange tr("fe_batch_submit");
    if (!ctx) return set_error(nullptr, FE_ERR_INVALID_ARG, "null context");
    if (!items || n_items <= 0) return set_error(ctx, FE_ERR_INVALID_ARG, "empty batch");
    if (n_items > (1 << 23)) return set_error(ctx, FE_ERR_INVALID_ARG, "too many batch items");
    for (int i = 0; i < n_items; ++i) {
        const fe_batch_item &it = items[i];
        fe_status st = fe_check_args(it.type, &it.args, &it.out);
        if (st != FE_OK) return set_error(ctx, st, "batch item " + std::to_string(i) + ": " + fe_last_error(nullptr));
        if (it.args.prec != FE_FP32_MIXED || it.args.memory != FE_MEM_DEVICE || it.out.memory != FE_MEM_DEVICE ||
            it.args.coords_layout != FE_LAYOUT_AOS || it.out.layout != FE_LAYOUT_AOS || it.out.packed ||
            it.args.coef_mode == FE_COEF_FUNCTION_U || it.args.ordering)
            return set_error(ctx, FE_ERR_UNSUPPORTED,
                             "batch items must be FE_FP32_MIXED, device memory, element-contiguous (AOS) in and out, not packed, coefficient arrays, ordering 0");
        if (it.args.n_elem >= (int64_t(1) << 40)) return set_error(ctx, FE_ERR_INVALID_ARG, "batch item too large");
    }
    cudaSetDevice(ctx->device);
    if (!ctx->batch) ctx->batch = new BatchCache();
    const size_t key = std::hash<std::string>()(
        std::string(reinterpret_cast<const char *>(items), sizeof(fe_batch_item) * size_t(n_items)));
    BatchPlan *pl = nullptr;
    for (auto it = ctx->batch->plans.begin(); it != ctx->batch->plans.end(); ++it) {
        if ((*it)->key == key && (*it)->items_bytes.size() == sizeof(fe_batch_item) * size_t(n_items) &&
            (*it)->pinned_block == ctx->batch_shape.block && (*it)->pinned_tpe == ctx->batch_shape.tpe &&
            (*it)->pinned_pers == ctx->batch_shape.persistent &&
            memcmp((*it)->items_bytes.data(), items, (*it)->items_bytes.size()) == 0) {
            pl = *it;
            ctx->batch->plans.erase(it);
            ctx->batch->plans.push_front(pl);
            break;
        }
    }
    if (!pl) {
        fe_status st = build_plan(ctx, items, n_items, key, pl);
        if (st != FE_OK) return st;
        ctx->batch->plans.push_front(pl);
        while (ctx->batch->plans.size() > 8) {
            cudaDeviceSynchronize();
            free_plan(ctx->batch->plans.back());
            ctx->batch->plans.pop_back();
        }
    }
    cudaError_t e = cudaGraphLaunch(pl->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_check(ctx, e, "cudaGraphLaunch(batch)");
    g_launches.fetch_add(uint64_t(plan_launches(pl)));
    return FE_OK;
}

}  // extern "C"
