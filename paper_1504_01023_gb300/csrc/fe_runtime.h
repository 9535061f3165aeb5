// Runtime internals shared by fe_runtime.cu, fe_batch.cu and fe_serve.cu.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "fe.h"
#include "fe_internal.h"

namespace fe {

// NVTX range over a host call (visible in Nsight Systems and any NVTX tool; a
// push and a pop into an empty stub when no tool is attached).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

extern std::atomic<uint64_t> g_launches;

// Device scratch of one launch sequence (fix-up list, its counter, status word).
struct Scratch {
    unsigned long long *fix_list = nullptr;
    unsigned int fix_cap = 0;
    unsigned int *fix_count = nullptr;
    int *status = nullptr;
};

struct Shape {
    int block = 0;          // elements per tile
    int persistent = 0;     // 1: grid = SMs x resident blocks, tiles strided
    int tpe = 1;            // threads per element (2: prisms, element-contiguous)
};

struct ServeState;          // fe_serve.cu
struct BatchCache;          // fe_batch.cu
struct BatchItemDev;
struct BatchSeg;

struct MeshRec {
    fe_elem_type type;
    int64_t n_elem;
    double *coords;         // SOA planes, stride n_elem, context-owned
    uint64_t bytes;
};

}  // namespace fe

struct fe_ctx {
    int device = 0;
    int sms = 0;
    int max_smem_optin = 0;
    std::string device_name;
    std::string last_error;
    std::mutex err_mu;
    fe_status async_error = FE_OK;

    fe::Scratch scratch;            // plain calls
    int *h_status = nullptr;        // pinned mirror for status reads

    // profiling
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;
    std::vector<cudaEvent_t> event_pool;

    // autotuner
    int autotune = 0;
    fe::Shape batch_shape{0, 1, 1};  // pinned shape of new batch plans (block 0: tuned or default)
    std::string tuning_cache_path;
    std::map<std::string, fe::Shape> shapes;

    // host-buffer pipeline
    cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
    void *stage[2][5] = {{nullptr}};
    uint64_t stage_bytes[2][5] = {{0}};

    // resident meshes
    std::mutex mesh_mu;
    std::unordered_map<int64_t, fe::MeshRec> meshes;
    int64_t next_mesh = 1;
    uint64_t hbm_budget = 0;
    std::atomic<uint64_t> hbm_used{0};

    fe::BatchCache *batch = nullptr;
    fe::ServeState *serve = nullptr;
    int serve_slots = 4;

    // injected faults (fe_ctx_inject_fault; test only)
    std::atomic<int64_t> fail_allocs{0};   // device allocations still to fail
    std::atomic<int64_t> skip_launches{0}; // main-kernel launches still to skip tiles
    int64_t skip_mod = 0;                  // their tile period
};

namespace fe {
fe_status set_error(fe_ctx *ctx, fe_status st, const std::string &msg);
fe_status cuda_check(fe_ctx *ctx, cudaError_t e, const char *what);
// Raise a kernel's dynamic shared-memory limit to at least `smem` bytes, never
// lower it; one process-wide record under a mutex, shared by every entry point
// that launches the kernel (ctx may be null).
fe_status set_smem_attr(fe_ctx *ctx, const void *k, int64_t smem);
// cudaMalloc for the context's own buffers; an injected allocation fault
// (fe_ctx_inject_fault) makes it fail with FE_ERR_OOM without allocating.
fe_status ctx_malloc(fe_ctx *ctx, void **p, size_t bytes, const char *what);
// True (and one injected fault used up) if the context's next allocation must fail.
bool take_alloc_fault(fe_ctx *ctx);
fe_status ensure_scratch(fe_ctx *ctx, Scratch &s, uint64_t n);
void free_scratch(Scratch &s);
// Launch main + fix-up kernels of one homogeneous set (device pointers).
// With `force`, that launch shape is used and the context's tuned shapes and
// profiling events are not touched (safe from the serving thread).
// x: the nodal input vector of the matrix-free output mode (fe_apply_*).
fe_status launch_set(fe_ctx *ctx, fe_elem_type type, const fe_elem_args *a, const fe_out *o, Scratch &s,
                     cudaStream_t st, const Shape *force = nullptr, const void *x = nullptr);
Shape default_shape(fe_elem_type type);
// Dynamically built batch (serving): device tables grown on demand, uploaded
// from pinned staging with stream-ordered copies, launched without a graph.
// One upload per launch: tile counters and the fix-up counter (zeroed), the item
// table and the segment table, staged in one pinned buffer.
struct DynBatch {
    unsigned char *d_tab = nullptr, *h_tab = nullptr;
    size_t cap_tab = 0;
    Scratch scratch;        // its fix-up list (the counter lives in the table)
};
fe_status dyn_batch_launch(fe_ctx *ctx, DynBatch &db, std::vector<BatchItemDev> &items, cudaStream_t st);
void dyn_batch_free(DynBatch &db);
int ns_of(fe_elem_type t);
int nq_of(fe_quad q);
int nc_of(fe_elem_type type, const fe_elem_args *a);
void batch_destroy(fe_ctx *ctx);
void serve_destroy(fe_ctx *ctx);
}  // namespace fe
